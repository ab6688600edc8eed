"""Batched solves (mr3_stemr_batched) against the oracle and against per-matrix solves."""
import numpy as np
import pytest

import oracle
import testmats as tm
from _checks import check_eigenpairs

pytestmark = pytest.mark.gpu


def _batched(sizes, seed0=900, rng="A", il=None, iu=None, vl=None, vu=None, fill=None):
    import torch
    import paper_1401_4950_gb300 as mr3
    n_off = np.zeros(len(sizes) + 1, dtype=np.int64)
    n_off[1:] = np.cumsum(sizes)
    d = np.empty(n_off[-1])
    e = np.zeros(n_off[-1])
    mats = []
    for b, n in enumerate(sizes):
        if fill is not None:
            db, eb = fill(b, n)
        else:
            db, eb = tm.random_uniform(n, seed0 + 2 * b, seed0 + 2 * b + 1)
        if n > 0:
            d[n_off[b]:n_off[b + 1]] = db
            e[n_off[b]:n_off[b + 1] - 1] = eb
        mats.append((db, eb))
    dt = torch.tensor(d, device="cuda")
    et = torch.tensor(e, device="cuda")
    m, w, Z, z_off, info = mr3.stemr_batched(n_off, dt, et, rng=rng, il=il, iu=iu, vl=vl, vu=vu)
    torch.cuda.synchronize()
    w = w.cpu().numpy()
    Z = Z.cpu().numpy()
    out = []
    for b, n in enumerate(sizes):
        k = int(m[b])
        wb = w[n_off[b]:n_off[b] + k]
        Zb = Z[z_off[b]:z_off[b] + n * k].reshape(k, n).T if n > 0 else np.zeros((0, 0))
        out.append((wb, Zb))
    return mats, out, info


def test_batched_uneven_sizes(cuda):
    sizes = [1, 2, 3, 17, 32, 100, 257, 1024, 5, 600]
    mats, out, info = _batched(sizes)
    for (d, e), (w, Z) in zip(mats, out):
        check_eigenpairs(d, e, w, Z)


def test_batched_empty_matrices(cuda):
    sizes = [0, 10, 0, 0, 7, 0]
    mats, out, _ = _batched(sizes)
    for (d, e), (w, Z) in zip(mats, out):
        if len(d):
            check_eigenpairs(d, e, w, Z)
        else:
            assert w.size == 0


def test_batched_equals_plain(cuda):
    import torch
    import paper_1401_4950_gb300 as mr3
    sizes = [50, 300, 129]
    mats, out, _ = _batched(sizes, seed0=77)
    for (d, e), (w, Z) in zip(mats, out):
        wp, Zp, _ = mr3.stemr(torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda"))
        assert np.array_equal(w, wp.cpu().numpy())
        assert np.array_equal(Z, Zp.cpu().numpy())


def test_batched_index_ranges(cuda):
    sizes = [40, 80, 120]
    il = [1, 10, 100]
    iu = [40, 20, 120]
    mats, out, _ = _batched(sizes, rng="I", il=il, iu=iu)
    for (d, e), (w, Z), a, b in zip(mats, out, il, iu):
        check_eigenpairs(d, e, w, Z, il=a, iu=b)


def test_batched_value_ranges(cuda):
    sizes = [60, 90]
    vl = [-0.5, 0.0]
    vu = [0.5, 2.0]
    mats, out, _ = _batched(sizes, rng="V", vl=vl, vu=vu)
    for (d, e), (w, Z), a, b in zip(mats, out, vl, vu):
        lo, hi = oracle.index_range(d, e, "V", vl=a, vu=b)
        assert w.size == max(hi - lo + 1, 0)
        if w.size:
            check_eigenpairs(d, e, w, Z, il=lo, iu=hi)


def test_batched_mixed_families(cuda):
    kinds = ["one_two_one", "wilkinson", "glued_wilkinson", "clement", "hermite", "random"]
    sizes = [200, 201, 126, 150, 180, 333]
    mats, out, info = _batched(sizes, fill=lambda b, n: tm.make(kinds[b], n, seed=5))
    for (d, e), (w, Z), k in zip(mats, out, kinds):
        check_eigenpairs(d, e, w, Z, vec_compare=False)


def test_batched_workload_sample(cuda):
    # the batched benchmark's workload shape: sizes uniform in [32, 1024], uniform(-1,1)
    sizes, n_off, d, e = tm.batched_random(64)
    mats, out, info = _batched(list(sizes), fill=lambda b, n: (d[n_off[b]:n_off[b + 1]],
                                                             e[n_off[b]:n_off[b + 1] - 1]))
    for (db, eb), (w, Z) in zip(mats, out):
        check_eigenpairs(db, eb, w, Z, vec_compare=False)


def test_batched_bench_step(cuda):
    # the n = 8192 step (1-2-1, Wilkinson W+, uniform(-1,1) seeds 201, 202) in one batched
    # call, as the benchmark times it: every matrix within the parity gates
    from _checks import check_eigenpairs
    mats = [tm.make("one_two_one", 8192), tm.make("wilkinson", 8192),
            tm.random_uniform(8192, 201, 202)]
    gates = [10.0, 10.0, 10.0]
    mats_out, out, info = _batched([8192, 8192, 8192], fill=lambda b, n: mats[b])
    for (d, e), (wb, Zb), gate in zip(mats, out, gates):
        check_eigenpairs(d, e, wb, Zb, orth_gate=gate, vec_compare=False)


@pytest.mark.parametrize("rng", ["A", "I"])
def test_batched_host_matches_device_call(cuda, rng):
    # mr3_stemr_batched_host (host buffers, copies inside the call) returns exactly what the
    # device call returns on the same packed batch, an empty matrix included
    import torch
    import paper_1401_4950_gb300 as mr3
    sizes = [37, 0, 300, 1, 129, 64]
    n_off = np.zeros(len(sizes) + 1, dtype=np.int64)
    n_off[1:] = np.cumsum(sizes)
    d = np.empty(n_off[-1])
    e = np.zeros(n_off[-1])
    for b, n in enumerate(sizes):
        db, eb = tm.random_uniform(n, 700 + 2 * b, 701 + 2 * b)
        d[n_off[b]:n_off[b + 1]] = db
        e[n_off[b]:n_off[b + 1] - 1] = eb
    kw = {}
    if rng == "I":
        kw = {"il": [max(1, n // 3) if n else 1 for n in sizes],
              "iu": [max(1, (2 * n) // 3) if n else 0 for n in sizes]}
        kw["il"] = [1 if n == 0 else a for a, n in zip(kw["il"], sizes)]
    m0, w0, Z0, z_off, _ = mr3.stemr_batched(n_off, torch.tensor(d, device="cuda"),
                                             torch.tensor(e, device="cuda"), rng=rng, **kw)
    torch.cuda.synchronize()
    m1, w1, Z1, z_off1, _ = mr3.stemr_batched_host(n_off, d, e, rng=rng, **kw)
    assert np.array_equal(m0, m1) and np.array_equal(z_off, z_off1)
    w0, Z0 = w0.cpu().numpy(), Z0.cpu().numpy()
    for b, n in enumerate(sizes):
        k = int(m0[b])
        assert np.array_equal(w1[n_off[b]:n_off[b] + k], w0[n_off[b]:n_off[b] + k])
        assert np.array_equal(Z1[z_off[b]:z_off[b] + n * k], Z0[z_off[b]:z_off[b] + n * k])
        if k:
            db, eb = d[n_off[b]:n_off[b + 1]], e[n_off[b]:n_off[b + 1] - 1]
            il = kw["il"][b] if kw else 1
            check_eigenpairs(db, eb, w1[n_off[b]:n_off[b] + k],
                             Z1[z_off[b]:z_off[b] + n * k].reshape(k, n).T, il=il,
                             iu=il + k - 1, vec_compare=False)
