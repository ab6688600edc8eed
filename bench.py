#!/usr/bin/env python3
"""Benchmark of the GB300 MRRR path: eigenpairs/s for all eigenpairs of n = 8192 FP64
symmetric tridiagonals (one 1-2-1, one Wilkinson W+ and one uniform(-1,1) matrix per
step, solved together by one mr3_stemr_batched call; --solver single times one mr3_stemr
call per matrix), with a live roofline of the dominant kernel, the CPU oracle timed
beside it, an end-to-end number (pinned host buffers copied in and out inside the timed
region), and SM clocks sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mr3|reference] [--config c2]

Under torchrun (N > 1) every rank solves its own copy of the step's matrices (the
problems are independent: weak scaling, no collective on the data path); the time is
the maximum over ranks.  `--impl reference` times the CPU oracle (bisection + inverse
iteration) on a bounded sample of the same workload, on rank 0 only.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import testmats as tm  # noqa: E402

EPS = 2.0 ** -53
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 pipe of a GB300: 152 SMs x 2 DFMA/clk (measured: 1.19 TFLOP/s at 1995 MHz) x 2 flop
# x 2070 MHz maximum SM clock.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12

CONFIGS = {
    "c1": {"workload": "plain MRRR, n=1000 uniform(-1,1) d and e, all eigenpairs, FP64",
           "mats": [("random", 1000, (101, 102))]},
    "c2": {"workload": "plain MRRR, n=8192 FP64, all eigenpairs, one matrix of each type per "
                       "step: 1-2-1 (d=2, e=-1), Wilkinson W+ (d_i=|i-(n-1)/2|, e=1), "
                       "uniform(-1,1) random d and e",
           "mats": [("one_two_one", 8192, None), ("wilkinson", 8192, None),
                    ("random", 8192, (201, 202))]},
}


def _workload(cfg, n_override=None):
    w = CONFIGS[cfg]["workload"]
    return w if not n_override else w + " (matrix order overridden: n=%d)" % n_override


def _matrices(cfg, n_override=None):
    out = []
    for kind, n, seeds in CONFIGS[cfg]["mats"]:
        n = n_override or n
        if kind == "random":
            d, e = tm.random_uniform(n, *seeds)
        else:
            d, e = tm.make(kind, n)
        out.append((kind, d, e))
    return out


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clk", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sms.append(float(p[1]))
                maxs.append(float(p[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxs) if maxs else None, "reasons": sorted(reasons),
                "samples": len(sms)}


# ------------------------------------------------------------------ CPU oracle legs

def oracle_sample(mats, per_matrix):
    """Oracle eigenpairs for `per_matrix` consecutive indices from the middle of each
    matrix's spectrum; returns (eigenpairs, seconds)."""
    import oracle
    t0 = time.perf_counter()
    count = 0
    for _, d, e in mats:
        n = len(d)
        il = max(1, n // 2 - per_matrix // 2)
        iu = min(n, il + per_matrix - 1)
        w = oracle.eigvals(d, e, il, iu)
        oracle.eigvecs(d, e, w)
        count += iu - il + 1
    return count, time.perf_counter() - t0


def calibrate_sample(mats, budget_s):
    per = 16
    while True:
        cnt, dt = oracle_sample(mats, per)
        if dt * 2.2 > budget_s or per >= 4096:
            return per, cnt, dt
        per *= 2


def cpu_baseline(mats, budget_s=15.0):
    per, cnt, dt = calibrate_sample(mats, budget_s)
    return {"value": cnt / dt, "unit": "eigenpairs/s", "cores": 1, "kind": "oracle",
            "sample": "%d consecutive mid-spectrum eigenpairs of each of the %d matrices "
                      "(bisection to full accuracy + inverse iteration with MGS), %.1f s, "
                      "single thread" % (per, len(mats), dt)}


def run_reference(args, cfg, rank):
    if rank != 0:
        return
    mats = _matrices(cfg, args.n)
    budget = max(2.0, 150.0 / (args.steps + args.warmup))
    per, _, _ = calibrate_sample(mats, budget)
    for _ in range(args.warmup):
        oracle_sample(mats, per)
    tot_cnt, tot_t = 0, 0.0
    for _ in range(args.steps):
        c, t = oracle_sample(mats, per)
        tot_cnt += c
        tot_t += t
    value = tot_cnt / tot_t
    line = {"impl": "reference", "metric": "eigenpairs/s (n=8192 all, FP64)", "value": value,
            "unit": "eigenpairs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": _workload(cfg, args.n),
                                            "sample_per_matrix": per},
            "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": 1,
                             "kind": "oracle",
                             "sample": "%d mid-spectrum eigenpairs per matrix per step" % per},
            "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ ranks

def max_over_ranks(ms, dist=None, device=None):
    """The slowest rank's time (the job ends when its last rank does); `ms` unchanged on
    one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms_per_step):
    """Whole-job throughput: every rank solves its own copy of the step's matrices (weak
    scaling), so the job processes world * units_per_rank units per step."""
    return world * units_per_rank / (ms_per_step / 1e3)


# ------------------------------------------------------------------ GPU leg

def run_gpu(args, cfg, rank, world):
    import torch
    import paper_1401_4950_gb300 as mr3
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    mats = _matrices(cfg, args.n)
    dev_mats = [(k, torch.tensor(d, device=dev), torch.tensor(e, device=dev)) for k, d, e in mats]
    units_per_step = sum(len(d) for _, d, _ in mats)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    opts = mr3.make_opts(profile=1, prec=mr3.DD if args.prec == "dd" else mr3.FP64)
    stream = torch.cuda.current_stream()
    # the step's matrices packed for one mr3_stemr_batched call (d and e with the same
    # offsets, the last e slot of each matrix unused)
    sizes = [len(d) for _, d, _ in mats]
    n_off = np.zeros(len(sizes) + 1, dtype=np.int64)
    n_off[1:] = np.cumsum(sizes)
    dcat_h = np.concatenate([np.asarray(d, dtype=np.float64) for _, d, _ in mats])
    ecat_h = np.concatenate([np.r_[np.asarray(e, dtype=np.float64), 0.0] for _, _, e in mats])
    dcat, ecat = torch.tensor(dcat_h, device=dev), torch.tensor(ecat_h, device=dev)

    def step():
        if args.solver == "single":
            infos = []
            for _, d, e in dev_mats:
                _, _, info = mr3.stemr(d, e, opts=opts)
                infos.append(info)
            return infos
        _, _, _, _, info = mr3.stemr_batched(n_off, dcat, ecat, opts=opts)
        return [info]

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    agg = {"kernel_ms": np.zeros(8), "kernel_launches": np.zeros(8, dtype=np.int64),
           "sturm_steps": 0, "shift_steps": 0, "twisted_steps": 0}
    last_infos = None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 (129 MB) flushed between timed steps
        ev[k][0].record(stream)
        infos = step()
        ev[k][1].record(stream)
        for inf in infos:
            agg["kernel_ms"] += np.array(inf["kernel_ms"])
            agg["kernel_launches"] += np.array(inf["kernel_launches"])
            for key in ("sturm_steps", "shift_steps", "twisted_steps"):
                agg[key] += inf[key]
        last_infos = infos
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = max_over_ranks(sum(step_ms), dist, dev)
    ms_per_step = tot_ms / args.steps
    value = job_value(units_per_step, world, ms_per_step)

    # ---- dominant kernel group and its roofline (FP64 pipe).  Algorithmic work per unit
    # (App. B recurrences): a Sturm-count step 5 flops (add, divide, multiply, FMA), a
    # dstqds trial step 5, a twisted-factorization step 5.5; the units are the steps the
    # library counts on the device, the time the group's CUDA events on its stream.
    g = agg["kernel_ms"]
    kl = agg["kernel_launches"]
    groups = {"k_bisect2 (root and child refinement)":
                  (g[2] + g[6], kl[2] + kl[6], agg["sturm_steps"], "Sturm step", 5.0),
              "k_rqi": (g[4], kl[4], agg["twisted_steps"], "twisted-factorization step", 5.5),
              "k_refine_ends + k_shift_*": (g[5], kl[5], agg["shift_steps"],
                                            "cluster-end Sturm / dstqds step", 5.0)}
    dom = max(groups, key=lambda k: groups[k][0])
    ms, launches, units, unit_name, fpu = groups[dom]
    achieved = (fpu * units / 1e12) / (ms / 1e3) if ms > 0 else 0.0
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "FP64 pipe: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz (no FP64 "
                               "figure in the measured peaks)",
                "algorithmic": {"unit": unit_name, "flops_per_unit": fpu,
                                "units_per_launch": units / max(launches, 1),
                                "ms_per_launch": ms / max(launches, 1)},
                "kernel_share": float(ms / max(g.sum(), 1e-9))}

    # ---- end to end through the public API: every step copies its inputs from pinned host
    # memory to the device, solves, and reads w and Z back into pinned host memory
    import ctypes
    L = mr3.lib()
    nmax = max(sizes)
    if args.solver == "single":
        Zh = torch.empty((nmax, nmax), dtype=torch.float64, pin_memory=True).numpy()
        wh = torch.empty(nmax, dtype=torch.float64, pin_memory=True).numpy()
        hbuf = []
        for _, d, e in mats:
            dh = torch.empty(len(d), dtype=torch.float64, pin_memory=True).numpy()
            eh = torch.empty(max(len(e), 1), dtype=torch.float64, pin_memory=True).numpy()
            dh[:] = d
            eh[: len(e)] = e
            hbuf.append((dh, eh))

        def e2e_step():
            for dh, eh in hbuf:
                n = len(dh)
                m = ctypes.c_int(0)
                rc = L.mr3_stemr_host(n, dh.ctypes.data_as(ctypes.c_void_p),
                                      eh.ctypes.data_as(ctypes.c_void_p), 0, 0.0, 0.0, 1, n,
                                      ctypes.byref(m), wh.ctypes.data_as(ctypes.c_void_p),
                                      Zh.ctypes.data_as(ctypes.c_void_p), n, ctypes.byref(opts),
                                      None, ctypes.c_void_p(stream.cuda_stream))
                assert rc in (0, 1, 2), rc
    else:
        # A serving loop: every step copies its inputs in from pinned host memory, solves,
        # and reads w and Z back into one of two pinned host buffers on a copy stream,
        # where the read of step k overlaps the solve of step k + 1 (the D2H of Z, 1.6 GB,
        # takes 8 ms at the C2C link's 193 GB/s but was seen at ~16 GB/s on a box whose host
        # was compacting memory).  The timed region ends when the last read is complete.
        dh = torch.tensor(dcat_h).pin_memory()
        eh = torch.tensor(ecat_h).pin_memory()
        zlen = int(sum(n * n for n in sizes))
        wh = [torch.empty(int(n_off[-1]), dtype=torch.float64, pin_memory=True) for _ in range(2)]
        Zh = [torch.empty(zlen, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        dd_, ed_ = torch.empty_like(dcat), torch.empty_like(ecat)
        copy_stream = torch.cuda.Stream(device=dev)
        e2e_k = [0]

        def e2e_step():
            slot = e2e_k[0] & 1
            e2e_k[0] += 1
            dd_.copy_(dh, non_blocking=True)
            ed_.copy_(eh, non_blocking=True)
            _, w, Z, _, _ = mr3.stemr_batched(n_off, dd_, ed_, opts=opts)
            solved = torch.cuda.Event()
            solved.record()
            copy_stream.wait_event(solved)
            with torch.cuda.stream(copy_stream):
                wh[slot].copy_(w[: wh[slot].numel()], non_blocking=True)
                Zh[slot].copy_(Z[:zlen], non_blocking=True)
            # the outputs stay allocated until the copy stream has read them; a pinned slot
            # is rewritten two steps later, after its previous read in copy-stream order
            w.record_stream(copy_stream)
            Z.record_stream(copy_stream)
    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne = max(2, min(args.steps, 5))
    for _ in range(ne):
        e2e_step()
    torch.cuda.synchronize()  # every step's read included
    e2e_s = (time.perf_counter() - t0) / ne
    h2d = sum(8 * (len(d) + len(e)) for _, d, e in mats)
    d2h = sum(8 * (len(d) + len(d) * len(d)) for _, d, _ in mats)
    e2e = {"value": world * units_per_step / e2e_s, "unit": "eigenpairs/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "steps": ne, "d2h": "copy stream, overlapping the next step's solve"
                              if args.solver != "single" else "inside mr3_stemr_host"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mats, budget_s=args.cpu_budget)
    info0 = last_infos[0] if last_infos else {}
    line = {"metric": "eigenpairs/s (n=8192 all, FP64)", "value": value, "unit": "eigenpairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload(cfg, args.n),
                       "n": [len(d) for _, d, _ in mats],
                       "matrices_per_step": len(mats), "l2": "flushed between steps "
                       "(256 MiB device write outside the per-step events)",
                       "parallelism": "replicas, one set of matrices per GPU",
                       "solver": args.solver,
                       "tree": "double-double (Ch. 5)" if args.prec == "dd" else "binary64"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(agg["kernel_launches"].sum()),
            "clocks": clk, "wall_s": wall,
            "solver": "mr3_stemr_batched over the step's matrices" if args.solver == "batched"
                      else "one mr3_stemr call per matrix",
            "solve_info": [dict(**{key: inf[key] for key in (
                "dmax", "largest_cluster", "nclusters", "new_rrr", "untested_rrr", "rqi_iters",
                "rqi_iters_max", "bisect_fallbacks", "sturm_steps", "shift_steps",
                "twisted_steps", "status")},
                kernel_ms=[round(x, 3) for x in inf["kernel_ms"]])
                for inf in (last_infos or [])],
            "step_ms": [round(x, 3) for x in step_ms]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_batched(args):
    """Batched workload: 4096 uniform(-1,1) tridiagonals with n_b uniform in [32, 1024], all
    eigenpairs, one mr3_stemr_batched call vs one mr3_stemr call per matrix (same stream,
    same accuracy).  Prints one JSON line (solves/s of both and their ratio)."""
    import torch
    import paper_1401_4950_gb300 as mr3
    dev = torch.device("cuda", 0)
    nb = args.batch
    sizes, n_off, d, e = tm.batched_random(nb)
    dt = torch.tensor(d, device=dev)
    et = torch.tensor(e, device=dev)
    opts = mr3.make_opts(profile=1)
    for _ in range(2):
        mr3.stemr_batched(n_off, dt, et, opts=opts)
    torch.cuda.synchronize()
    reps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(reps):
        m, w, Z, z_off, info = mr3.stemr_batched(n_off, dt, et, opts=opts)
    torch.cuda.synchronize()
    tb = (time.perf_counter() - t0) / reps
    # per-matrix plain launches on the same data
    views = [(dt[n_off[b]:n_off[b + 1]], et[n_off[b]:n_off[b + 1]]) for b in range(nb)]
    for b in range(min(nb, 8)):
        mr3.stemr(*views[b])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b in range(nb):
        mr3.stemr(*views[b])
    torch.cuda.synchronize()
    tp = time.perf_counter() - t0
    line = {"metric": "batched solves/s (4096 tridiagonals, n in [32,1024], all eigenpairs, FP64)",
            "value": nb / tb, "unit": "solves/s", "per_matrix_value": nb / tp,
            "batched_over_per_matrix": tp / tb, "batched_ms": 1e3 * tb, "per_matrix_ms": 1e3 * tp,
            "eigenpairs": int(n_off[-1]), "kernel_ms": [round(x, 3) for x in info["kernel_ms"]],
            "dmax": info["dmax"], "nclusters": info["nclusters"], "rqi_iters": info["rqi_iters"]}
    print(json.dumps(line), flush=True)


def run_backward(args):
    """Backward vs forward at n = 4096 (uniform(-1,1) d and e, all eigenpairs): loss
    sum(g . lambda) + sum(G o Z), g and G standard normal.  Prints one JSON line."""
    import torch
    import paper_1401_4950_gb300 as mr3
    dev = torch.device("cuda", 0)
    n = args.n_bwd
    d, e = tm.random_uniform(n, 501, 502)
    g = torch.tensor(tm.normal(503, n), device=dev)
    G = torch.tensor(tm.normal(504, n * n).reshape(n, n), device=dev).t().contiguous().t()
    dt, et = torch.tensor(d, device=dev), torch.tensor(e, device=dev)
    for _ in range(2):
        w, Z, _ = mr3.stemr(dt, et)
        mr3.backward(w, Z, g, G)
    torch.cuda.synchronize()
    reps = max(1, args.steps)
    t0 = time.perf_counter()
    for _ in range(reps):
        w, Z, _ = mr3.stemr(dt, et)
    torch.cuda.synchronize()
    tf = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        dd, de = mr3.backward(w, Z, g, G)
    torch.cuda.synchronize()
    tb = (time.perf_counter() - t0) / reps
    print(json.dumps({"metric": "backward / forward time (n=%d, all eigenpairs, FP64)" % n,
                      "value": tb / tf, "unit": "ratio", "forward_ms": 1e3 * tf,
                      "backward_ms": 1e3 * tb}), flush=True)


def _gpu_gates(d, e, w, Z, tnorm):
    """Scaled residual max ||T z - lambda z|| / (n eps ||T||) and orthogonality
    max |Z^T Z - I| / (n eps), computed with plain torch operations on the device."""
    import torch
    n = d.shape[0]
    TZ = d[:, None] * Z
    TZ[:-1] += e[:n - 1, None] * Z[1:]
    TZ[1:] += e[:n - 1, None] * Z[:-1]
    R = TZ - Z * w[None, :]
    resid = torch.linalg.vector_norm(R, dim=0).max().item() / (n * EPS * tnorm)
    G = Z.T @ Z
    G.diagonal().sub_(1.0)
    orth = G.abs().max().item() / (n * EPS)
    return resid, orth


def run_subset(args):
    """Subset workload: eigenpairs 8001..12000 of the n = 20000 glued Wilkinson matrix (W21+
    blocks glued by 1e-8), binary64 tree vs double-double tree.  Prints one JSON line."""
    import torch
    import paper_1401_4950_gb300 as mr3
    dev = torch.device("cuda", 0)
    n, il, iu = 20000, 8001, 12000
    d, e = tm.make("glued_wilkinson", n)
    dt, et = torch.tensor(d, device=dev), torch.tensor(e, device=dev)
    w1, _, _ = mr3.stemr(dt, et, rng="I", il=1, iu=1)
    wn, _, _ = mr3.stemr(dt, et, rng="I", il=n, iu=n)
    tnorm = max(abs(w1.item()), abs(wn.item()))
    out = {"metric": "eigenpairs/s (n=20000 glued Wilkinson, eigenpairs 8001..12000)",
           "unit": "eigenpairs/s", "config": {"workload": "MRRR subset, n=20000 glued W21+ "
                                              "(e=1e-8 at joins), il=8001, iu=12000"}}
    for name, prec in (("fp64", mr3.FP64), ("dd", mr3.DD)):
        opts = mr3.make_opts(prec=prec, profile=1)
        for _ in range(2):
            mr3.stemr(dt, et, rng="I", il=il, iu=iu, opts=opts)
        torch.cuda.synchronize()
        reps = max(1, args.steps)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(reps):
            w, Z, info = mr3.stemr(dt, et, rng="I", il=il, iu=iu, opts=opts)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        resid, orth = _gpu_gates(dt, et, w, Z, tnorm)
        out[name] = {"value": (iu - il + 1) / (ms * 1e-3), "ms": ms, "resid": resid,
                     "orth": orth, "dmax": info["dmax"], "nclusters": info["nclusters"],
                     "largest_cluster": info["largest_cluster"],
                     "rqi_iters": info["rqi_iters"], "bisect_fallbacks": info["bisect_fallbacks"],
                     "status": info["status"],
                     "kernel_ms": [round(x, 3) for x in info["kernel_ms"]]}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mr3", choices=["mr3", "reference"])
    ap.add_argument("--config", default="c2", choices=sorted(CONFIGS))
    ap.add_argument("--n", type=int, default=None,
                    help="matrix order instead of the config's (smaller cases for ncu captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--batched", action="store_true",
                    help="time the batched workload (one call vs per-matrix calls) instead")
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--backward", action="store_true",
                    help="time the backward pass against the forward instead")
    ap.add_argument("--n-bwd", type=int, default=4096)
    ap.add_argument("--solver", default="batched", choices=["batched", "single"],
                    help="the step's matrices in one mr3_stemr_batched call, or one mr3_stemr "
                         "call each")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "dd"],
                    help="representation tree in binary64 or double-double (Ch. 5)")
    ap.add_argument("--subset", action="store_true",
                    help="time the n=20000 glued Wilkinson subset, binary64 vs double-double")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, args.config, rank)
        return
    if args.batched:
        run_batched(args)
        return
    if args.backward:
        run_backward(args)
        return
    if args.subset:
        run_subset(args)
        return
    run_gpu(args, args.config, rank, world)


if __name__ == "__main__":
    main()
