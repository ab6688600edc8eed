"""Launch-shape autotuner for the MRRR solver.

Two launch parameters of the solve do not change what it computes, only how the work is
spread over the GPU:

* ``bisect_warps``: the warps per SM the eigenvalue bisection aims for, which sets the
  lanes per eigenvalue of the multisection (Alg. Bisection run on several points of an
  interval at once): few eigenvalues get many lanes each, many eigenvalues get one;
* ``rqi_team``: the lanes that share one singleton in the twisted-factorization RQI
  (Alg. Getvec): teams of 8 finish one vector with less latency, teams of 2 keep more
  singletons in flight.

The library picks both from the size of the work by fixed rules.  ``tune`` times every
candidate pair on a given batch (CUDA events on the calling stream), rejects any whose
result misses the accuracy gates (scaled residual and orthogonality at most 10, the
bounds the method is held to), and stores the fastest under the batch's size class in a
JSON cache (one entry per device name and library build).  ``tuned_opts`` returns the
options for a batch from that cache, or the library's defaults for a size class that was
never tuned.

The tuner only calls the solver's public entry points; the gates use plain tensor
operations on the device.
"""
from __future__ import annotations

import json
import math
import os
import threading

import numpy as np

from . import build_lib

# (rqi_team, bisect_warps); 0 leaves the parameter to the library's rule
CANDIDATES = ((0, 0), (2, 24), (2, 48), (2, 64), (8, 24), (8, 48), (8, 64))
GATE = 10.0
_EPS = 2.0 ** -53
_lock = threading.Lock()


def cache_path() -> str:
    """The JSON cache: $MR3_AUTOTUNE_CACHE, else autotune.json in the build folder."""
    return os.environ.get("MR3_AUTOTUNE_CACHE") or os.path.join(build_lib.BUILD, "autotune.json")


def _pow2(x: int) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(int(x), 1)))))


def size_class(sizes, tree_opts=None) -> str:
    """Bucket of a batch: the number of matrices, the largest order and the total order,
    each rounded up to a power of two, plus the tree options that change the work (the
    absolute-gap split, the e-representation) when set."""
    sizes = np.asarray(sizes, dtype=np.int64).ravel()
    if sizes.size == 0:
        return "empty"
    key = "nmat%d_nmax%d_rows%d" % (_pow2(sizes.size), _pow2(int(sizes.max())),
                                    _pow2(int(sizes.sum())))
    for name in sorted(tree_opts or {}):
        if tree_opts[name]:
            key += "_%s%d" % (name, int(tree_opts[name]))
    return key


def _lib_fingerprint() -> str:
    import hashlib
    from . import lib
    lib()  # built and loaded
    h = hashlib.sha256()
    with open(build_lib.LIB, "rb") as f:
        for chunk in iter(lambda: f.read(1 << 20), b""):
            h.update(chunk)
    return h.hexdigest()[:16]


def _device_key() -> str:
    """Device name and library build: a rebuilt library is tuned afresh."""
    import torch
    return "%s|%s" % (torch.cuda.get_device_name(), _lib_fingerprint())


def _load(path=None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def _store(entry_key: str, cls: str, entry: dict, path=None) -> None:
    path = path or cache_path()
    with _lock:
        data = _load(path)
        data.setdefault(entry_key, {})[cls] = entry
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def lookup(sizes, path=None, tree_opts=None):
    """The cached choice for a batch of these orders on this device, or None."""
    return _load(path).get(_device_key(), {}).get(size_class(sizes, tree_opts))


def choose(timings: dict, passed: dict):
    """The fastest candidate that met the gates: timings and passed map a candidate key
    'team,warps' to its median milliseconds and to its gate verdict.  None if none
    passed."""
    best = None
    for key, ms in timings.items():
        if not passed.get(key):
            continue
        if best is None or ms < timings[best]:
            best = key
    return best


def _key(team, warps) -> str:
    return "%d,%d" % (team, warps)


def _gates(n_off, d, e, w, Z, z_off, check_max):
    """max over the checked matrices of the scaled residual and orthogonality; the largest
    matrices of the batch are checked (at most check_max of them)."""
    import torch
    sizes = np.diff(n_off)
    order = np.argsort(-sizes, kind="stable")[:check_max]
    worst_r = worst_o = 0.0
    for b in order:
        n = int(sizes[b])
        if n == 0:
            continue
        db = d[n_off[b]:n_off[b] + n]
        eb = e[n_off[b]:n_off[b] + n]
        wb = w[n_off[b]:n_off[b] + n]
        Zb = Z[z_off[b]:z_off[b] + n * n].view(n, n).t()  # column j = eigenvector j
        TZ = db[:, None] * Zb
        if n > 1:
            TZ[:-1] += eb[:n - 1, None] * Zb[1:]
            TZ[1:] += eb[:n - 1, None] * Zb[:-1]
        tn = max(abs(float(wb[0])), abs(float(wb[-1])), 1e-300)
        r = torch.linalg.vector_norm(TZ - Zb * wb[None, :], dim=0).max().item() / (n * _EPS * tn)
        G = Zb.T @ Zb
        G.diagonal().sub_(1.0)
        o = G.abs().max().item() / (n * _EPS)
        worst_r, worst_o = max(worst_r, r), max(worst_o, o)
    return worst_r, worst_o


def tune(n_off, d, e, reps=3, warmup=1, candidates=CANDIDATES, check_max=4, store=True,
         path=None, stream=None, tree_opts=None):
    """Time every candidate launch shape on the packed batch (n_off host offsets; d, e
    device float64 tensors packed as for stemr_batched, all eigenpairs in binary64),
    store the fastest one that meets the gates, and return the record:
    {"class", "rqi_team", "bisect_warps", "ms", "timings", "gates"}, gates holding each
    candidate's [residual, orthogonality, status].  tree_opts (abs_split, erep) are passed
    to every solve and are part of the size class."""
    import torch
    from . import make_opts, stemr_batched
    n_off = np.ascontiguousarray(n_off, dtype=np.int64)
    s = stream if stream is not None else torch.cuda.current_stream()
    timings, passed, gates = {}, {}, {}
    for team, warps in candidates:
        o = make_opts(rqi_team=team, bisect_warps=warps, **(tree_opts or {}))
        for _ in range(max(warmup, 0)):
            stemr_batched(n_off, d, e, opts=o, stream=s)
        ms = []
        res = None
        for _ in range(max(reps, 1)):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            res = stemr_batched(n_off, d, e, opts=o, stream=s)
            b.record(s)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        _, w, Z, z_off, info = res
        r, q = _gates(n_off, d, e, w, Z, z_off, check_max)
        k = _key(team, warps)
        timings[k] = float(np.median(ms))
        gates[k] = [round(r, 3), round(q, 3), int(info["status"])]
        # status 1 (a representation accepted by least growth) is a warning: the gates decide
        passed[k] = bool(info["status"] in (0, 1) and r <= GATE and q <= GATE)
        del res, w, Z
    best = choose(timings, passed)
    if best is None:
        team, warps = 0, 0
    else:
        team, warps = (int(x) for x in best.split(","))
    rec = {"class": size_class(np.diff(n_off), tree_opts), "rqi_team": team, "bisect_warps": warps,
           "ms": timings.get(best), "timings": timings, "gates": gates}
    if store and best is not None:
        _store(_device_key(), rec["class"], rec, path)
    return rec


def tuned_opts(sizes, path=None, **kw):
    """make_opts(**kw) with the cached launch shape for a batch of these orders (the
    library's defaults when the class was never tuned on this device)."""
    from . import make_opts
    rec = lookup(sizes, path, {k: kw[k] for k in ("abs_split", "erep") if kw.get(k)})
    if rec is not None:
        kw.setdefault("rqi_team", int(rec.get("rqi_team", 0)))
        kw.setdefault("bisect_warps", int(rec.get("bisect_warps", 0)))
    return make_opts(**kw)
