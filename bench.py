#!/usr/bin/env python3
"""Benchmark of the GB300 MRRR path.

The headline line times all eigenpairs of n = 8192 FP64 symmetric tridiagonals (one
1-2-1, one Wilkinson W+ and one uniform(-1,1) matrix per step, solved together by one
mr3_stemr_batched call; --solver single times one mr3_stemr call per matrix), with the
accuracy of each matrix's result, a live roofline of the dominant kernel group, the CPU
oracle timed beside it, an end-to-end number through mr3_stemr_batched_host (host buffers
copied in and out inside the timed call), and SM clocks sampled during the timed region.
The same line carries the other parts of the metric: batched solves/s (4096 matrices of
orders 32..1024, one call against per-matrix calls), backward / forward time at n = 4096,
and the n = 20000 glued Wilkinson subset with the binary64 and the double-double tree.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mr3|reference] [--config c2]
                  [--no-extras]

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
# A binary64 division occupies the FP64 pipe for about 10 DFMA issue slots (measured with
# dependent a/b chains against FMA chains): in the divide-weighted count a division is
# 20 flop-equivalents at the pipe's peak instead of 1 flop.
DIV_FLOP_EQ = 20.0
# Oracle sample of both CPU legs (the cpu_baseline of the headline line and the
# reference arm): consecutive mid-spectrum eigenpairs per matrix.
ORACLE_SAMPLE = 256
# DRAM traffic per launch of the dominant kernel group, from an ncu capture of the same
# workload (dram__bytes_read.sum + dram__bytes_write.sum, summed over the group's launches
# of one step and divided by their number), valid only while the kernel source it was
# taken on is unchanged: source file, its sha256 prefix at capture time, and the summary
# under profiles/ that holds the counters.
# The capture's RQI team size is part of its validity (0: the library's own rule).
TRAFFIC = {"k_rqi": {"bytes_per_launch": 3.189e9,
                     "source": "paper_1401_4950_gb300/csrc/mr3_rqi.cu", "sha": "ac3e79a3631ebebd",
                     "profile": "profiles/k_rqi_traffic_step_n8192.md", "rqi_team": 0}}

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

def host_info():
    """The host the CPU legs ran on: logical CPUs and the CPU model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


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


def _sample_text(per, nmat):
    return ("%d consecutive mid-spectrum eigenpairs of each of the %d matrices (bisection to "
            "full accuracy + inverse iteration with MGS), single thread" % (per, nmat))


def cpu_baseline(mats, reps=2):
    """The oracle on the same sample as the reference arm, timed `reps` times (~10 s)."""
    cnt, tot = 0, 0.0
    for _ in range(reps):
        c, t = oracle_sample(mats, ORACLE_SAMPLE)
        cnt += c
        tot += t
    return {"value": cnt / tot, "unit": "eigenpairs/s", "cores": 1, "kind": "oracle",
            "sample": _sample_text(ORACLE_SAMPLE, len(mats)) + ", %d repetitions, %.1f s" % (reps, tot),
            "host": host_info()}


def run_reference(args, cfg, rank):
    if rank != 0:
        return
    mats = _matrices(cfg, args.n)
    for _ in range(args.warmup):
        oracle_sample(mats, ORACLE_SAMPLE)
    tot_cnt, tot_t = 0, 0.0
    for _ in range(args.steps):
        c, t = oracle_sample(mats, ORACLE_SAMPLE)
        tot_cnt += c
        tot_t += t
    value = tot_cnt / tot_t
    line = {"impl": "reference", "metric": "eigenpairs/s (n=8192 all, FP64)", "value": value,
            "unit": "eigenpairs/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": _workload(cfg, args.n),
                                            "sample_per_matrix": ORACLE_SAMPLE},
            "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": 1,
                             "kind": "oracle", "sample": _sample_text(ORACLE_SAMPLE, len(mats)),
                             "host": host_info()},
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


# ------------------------------------------------------------------ accuracy on the device

def gpu_gates(d, e, w, Z, tnorm):
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


def _source_sha(path):
    import hashlib
    return hashlib.sha256(open(os.path.join(ROOT, path), "rb").read()).hexdigest()[:16]


def traffic_for(kernel, rqi_team=0):
    """DRAM bytes per launch of `kernel` from its capture, or None when the kernel's source
    changed after the capture, the step runs another RQI team size than the capture did,
    or no capture exists."""
    t = TRAFFIC.get(kernel)
    if not t or _source_sha(t["source"]) != t["sha"]:
        return None
    if kernel == "k_rqi" and t.get("rqi_team", 0) != rqi_team:
        return None
    return t["bytes_per_launch"]


def autotuned(n_off, d, e, args, tree_opts=None):
    """The launch shape for this batch: tuned now (untimed, before the warm-up) unless
    --no-autotune, else the library's rules.  Returns (rqi_team, bisect_warps, record)."""
    if args.no_autotune or args.prec == "dd":
        return 0, 0, None
    from paper_1401_4950_gb300 import autotune
    rec = autotune.tune(n_off, d, e, reps=2, warmup=1, tree_opts=tree_opts)
    return rec["rqi_team"], rec["bisect_warps"], rec


# ------------------------------------------------------------------ GPU legs

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
    stream = torch.cuda.current_stream()
    # the step's matrices packed for one mr3_stemr_batched call (d and e with the same
    # offsets, the last e slot of each matrix unused)
    sizes = [len(d) for _, d, _ in mats]
    n_off = np.zeros(len(sizes) + 1, dtype=np.int64)
    n_off[1:] = np.cumsum(sizes)
    dcat_h = np.concatenate([np.asarray(d, dtype=np.float64) for _, d, _ in mats])
    ecat_h = np.concatenate([np.r_[np.asarray(e, dtype=np.float64), 0.0] for _, _, e in mats])
    dcat, ecat = torch.tensor(dcat_h, device=dev), torch.tensor(ecat_h, device=dev)
    tree_flags = {"abs_split": int(args.abs_split), "erep": int(args.erep)}
    team, bwarps, tuned = autotuned(n_off, dcat, ecat, args, tree_flags)
    opts = mr3.make_opts(profile=1, prec=mr3.DD if args.prec == "dd" else mr3.FP64,
                         rqi_team=team, bisect_warps=bwarps, **tree_flags)

    def step():
        """One step; returns the solver statistics and each matrix's (w, Z) on the device."""
        if args.solver == "single":
            infos, res = [], []
            for _, d, e in dev_mats:
                w, Z, info = mr3.stemr(d, e, opts=opts)
                infos.append(info)
                res.append((w, Z))
            return infos, res
        _, w, Z, z_off, info = mr3.stemr_batched(n_off, dcat, ecat, opts=opts)
        res = []
        for b, n in enumerate(sizes):
            res.append((w[n_off[b]:n_off[b] + n],
                        Z[z_off[b]:z_off[b] + n * n].view(n, n).t()))
        return [info], res

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    agg = {"kernel_ms": np.zeros(8), "kernel_launches": np.zeros(8, dtype=np.int64),
           "sturm_steps": 0, "shift_steps": 0, "twisted_steps": 0}
    last = None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))  # L2 (129 MB) flushed between timed steps
        ev[k][0].record(stream)
        infos, res = step()
        ev[k][1].record(stream)
        for inf in infos:
            agg["kernel_ms"] += np.array(inf["kernel_ms"])
            agg["kernel_launches"] += np.array(inf["kernel_launches"])
            for key in ("sturm_steps", "shift_steps", "twisted_steps"):
                agg[key] += inf[key]
        last = (infos, res)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = max_over_ranks(sum(step_ms), dist, dev)
    ms_per_step = tot_ms / args.steps
    value = job_value(units_per_step, world, ms_per_step)

    # ---- accuracy of the last timed step's results (outside the timed region): the
    # spec gates, residual and orthogonality scaled by n eps ||T|| and n eps
    accuracy = []
    for (kind, d, e), (w, Z) in zip(dev_mats, last[1]):
        tn = max(abs(w[0].item()), abs(w[-1].item()))
        r, o = gpu_gates(d, e, w, Z, tn)
        accuracy.append({"matrix": kind, "n": int(d.shape[0]), "resid": round(r, 4),
                         "orth": round(o, 4)})
    del last

    # ---- dominant kernel group and its roofline (FP64 pipe).  Algorithmic work per unit
    # (App. B recurrences): a Sturm-count step 5 flops (add, divide, multiply, FMA), a
    # dstqds trial step 5, a twisted-factorization step 5.5, each with one division; the
    # units are the steps the library counts on the device, the time the group's CUDA
    # events on its stream.  The divide-weighted count charges each division at its
    # measured cost on the pipe (DIV_FLOP_EQ flop-equivalents).
    g = agg["kernel_ms"]
    kl = agg["kernel_launches"]
    groups = {"k_bisect2 (root and child refinement)":
                  (g[2] + g[6], kl[2] + kl[6], agg["sturm_steps"], "Sturm step", 5.0, "k_bisect2"),
              "k_rqi": (g[4], kl[4], agg["twisted_steps"], "twisted-factorization step", 5.5,
                        "k_rqi"),
              "k_refine_ends + k_shift_*": (g[5], kl[5], agg["shift_steps"],
                                            "cluster-end Sturm / dstqds step", 5.0, "k_shift")}
    dom = max(groups, key=lambda k: groups[k][0])
    ms, launches, units, unit_name, fpu, kname = groups[dom]
    fpu_w = fpu - 1.0 + DIV_FLOP_EQ
    achieved = (fpu * units / 1e12) / (ms / 1e3) if ms > 0 else 0.0
    achieved_w = (fpu_w * units / 1e12) / (ms / 1e3) if ms > 0 else 0.0
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": traffic_for(kname, team),
                "frac_divide_weighted": achieved_w / FP64_PEAK_TFLOPS,
                "peak_source": "FP64 pipe: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz, from unit "
                               "counts and the maximum clock (MEASURED_PEAKS.json has no FP64 "
                               "figure; a microbenchmark measured 1.19 TFLOP/s at 1995 MHz)",
                "algorithmic": {"unit": unit_name, "flops_per_unit": fpu,
                                "flops_per_unit_divide_weighted": fpu_w,
                                "units_per_launch": units / max(launches, 1),
                                "ms_per_launch": ms / max(launches, 1),
                                "z_bytes_per_step": int(8 * sum(n * n + n for n in sizes))},
                "kernel_share": float(ms / max(g.sum(), 1e-9))}
    if TRAFFIC.get(kname):
        roofline["traffic_source"] = {k: TRAFFIC[kname][k] for k in ("profile", "sha", "source")}

    # ---- end to end through the C ABI on host buffers: every step is one
    # mr3_stemr_batched_host call, which copies d and e in from pinned host memory, solves,
    # and copies w and Z back into pinned host memory before returning.  The library's
    # memory pool is handed back to the driver first, so that these calls find the pool a
    # fresh process has after its first call, not the blocks the launch-shape tuning and
    # the headline steps left in it.
    torch.cuda.synchronize()
    mr3.release_memory()
    dh = torch.tensor(dcat_h).pin_memory()
    eh = torch.tensor(ecat_h).pin_memory()
    zlen = int(sum(n * n for n in sizes))
    wh = torch.empty(int(n_off[-1]), dtype=torch.float64).pin_memory()
    Zh = torch.empty(zlen, dtype=torch.float64).pin_memory()
    e2e_opts = mr3.make_opts(prec=opts.prec, rqi_team=team, bisect_warps=bwarps, **tree_flags)

    def e2e_step():
        if args.solver == "single":
            for _, d, e in mats:
                mr3.stemr_host(d, e, opts=e2e_opts)
        else:
            mr3.stemr_batched_host(n_off, dh, eh, opts=e2e_opts, out=(wh, Zh))

    e2e_step()
    torch.cuda.synchronize()
    ne = max(2, min(args.steps, 5))
    e2e_ms = []
    for _ in range(ne):
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_s = sum(e2e_ms) / ne / 1e3
    h2d = 8 * (len(dcat_h) + len(ecat_h))
    d2h = 8 * (int(n_off[-1]) + zlen)
    e2e = {"value": world * units_per_step / e2e_s, "unit": "eigenpairs/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": ne,
           "ms_all": [round(x, 3) for x in e2e_ms],
           "api": "mr3_stemr_batched_host (C ABI, pinned host buffers, copies inside the call)"
                  if args.solver != "single" else "mr3_stemr_host per matrix (C ABI)"}
    del dh, eh, wh, Zh

    extras = {}
    if not args.no_extras and world == 1:
        extras["batched"] = batched_leg(args)
        extras["backward"] = backward_leg(args)
        extras["subset"] = subset_leg(args)
        extras["left_subsets"] = left_subset_leg(args)
        if args.prec == "fp64" and not args.abs_split:
            extras["abs_split"] = abs_split_leg(args, cfg)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mats)
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
                       "tree": "double-double (Ch. 5)" if args.prec == "dd" else "binary64",
                       "launch_shape": {"rqi_team": team, "bisect_warps": bwarps,
                                        "autotune": tuned},
                       "tree_options": tree_flags},
            "accuracy": accuracy,
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
                for inf in infos],
            "step_ms": [round(x, 3) for x in step_ms]}
    line.update(extras)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def batched_leg(args):
    """Batched workload: 4096 uniform(-1,1) tridiagonals with n_b uniform in [32, 1024], all
    eigenpairs, one mr3_stemr_batched call against one mr3_stemr call per matrix on the same
    stream (same kernels, same accuracy); median of the timed calls."""
    import torch
    import paper_1401_4950_gb300 as mr3
    dev = torch.device("cuda", torch.cuda.current_device())
    nb = args.batch
    sizes, n_off, d, e = tm.batched_random(nb)
    dt = torch.tensor(d, device=dev)
    et = torch.tensor(e, device=dev)
    tree_flags = {"abs_split": int(args.abs_split), "erep": int(args.erep)}
    team, bwarps, tuned = autotuned(n_off, dt, et, args, tree_flags)
    # the level loop in one CUDA graph (kernel_ms[3] then holds the levels' time)
    opts = mr3.make_opts(profile=1, rqi_team=team, bisect_warps=bwarps, graph=1, **tree_flags)
    for _ in range(2):
        mr3.stemr_batched(n_off, dt, et, opts=opts)
    torch.cuda.synchronize()
    reps = max(3, min(args.steps, 5))
    tb = []
    for _ in range(reps):
        a, b = _events()
        a.record()
        m, w, Z, z_off, info = mr3.stemr_batched(n_off, dt, et, opts=opts)
        b.record()
        torch.cuda.synchronize()
        tb.append(a.elapsed_time(b))
        if len(tb) < reps:
            del w, Z
    tbm = statistics.median(tb)
    # the same solve with the host-driven level loop (a counter read-back per level): its
    # time, and whether the outputs are identical
    hopts = mr3.make_opts(rqi_team=team, bisect_warps=bwarps, graph=-1, **tree_flags)
    th = []
    for _ in range(2):
        a, b = _events()
        a.record()
        _, wh, Zh, _, ih = mr3.stemr_batched(n_off, dt, et, opts=hopts)
        b.record()
        torch.cuda.synchronize()
        th.append(a.elapsed_time(b))
    same = bool(torch.equal(w, wh) and torch.equal(Z, Zh))
    del w, Z, wh, Zh
    loop = {"graph_levels": info["graph_levels"], "graph_runs": info["graph_runs"],
            "arena_peak_gb": round(8 * info["graph_pool_peak"] / 1e9, 2),
            "host_loop_ms": min(th), "identical_to_host_loop": same,
            "note": "one mr3_stemr_batched call: prologue and root bisection, the tree's "
                    "levels as one CUDA graph launch (no counter read-back between levels), "
                    "output ordering"}
    if args.no_per_matrix:
        return {"metric": "batched solves/s (4096 tridiagonals, n in [32,1024], all eigenpairs, "
                          "FP64)", "value": nb / (tbm / 1e3), "unit": "solves/s",
                "batched_ms": tbm, "batched_ms_all": tb,
                "kernel_ms": [round(x, 3) for x in info["kernel_ms"]], "dmax": info["dmax"],
                "nclusters": info["nclusters"], "level_loop": loop}
    # the per-matrix loop runs with the library's own launch-shape rules
    popts = mr3.make_opts(**tree_flags)
    views = [(dt[n_off[b]:n_off[b + 1]], et[n_off[b]:n_off[b + 1]]) for b in range(nb)]
    for b in range(min(nb, 8)):
        mr3.stemr(*views[b], opts=popts)
    torch.cuda.synchronize()
    a, b_ = _events()
    a.record()
    for b in range(nb):
        mr3.stemr(*views[b], opts=popts)
    b_.record()
    torch.cuda.synchronize()
    tp = a.elapsed_time(b_)
    return {"metric": "batched solves/s (4096 tridiagonals, n in [32,1024], all eigenpairs, FP64)",
            "value": nb / (tbm / 1e3), "unit": "solves/s", "per_matrix_value": nb / (tp / 1e3),
            "batched_over_per_matrix": tp / tbm, "batched_ms": tbm, "batched_ms_all": tb,
            "per_matrix_ms": tp, "eigenpairs": int(n_off[-1]),
            "kernel_ms": [round(x, 3) for x in info["kernel_ms"]], "dmax": info["dmax"],
            "nclusters": info["nclusters"], "rqi_iters": info["rqi_iters"],
            "level_loop": loop,
            "launch_shape": {"rqi_team": team, "bisect_warps": bwarps, "autotune": tuned},
            "tree_options": tree_flags,
            "config": "sizes seed 401; matrix b: d seed 402+2b, e seed 403+2b"}


def abs_split_leg(args, cfg):
    """The headline step again with the root classification amended by absolute gaps
    (opts.abs_split): its throughput, the accuracy gates of each matrix and the number of
    representations accepted by least growth (untested), which the option can raise."""
    import torch
    import paper_1401_4950_gb300 as mr3
    dev = torch.device("cuda", torch.cuda.current_device())
    mats = _matrices(cfg, args.n)
    sizes = [len(d) for _, d, _ in mats]
    n_off = np.zeros(len(sizes) + 1, dtype=np.int64)
    n_off[1:] = np.cumsum(sizes)
    dcat = torch.tensor(np.concatenate([np.asarray(d, dtype=np.float64) for _, d, _ in mats]),
                        device=dev)
    ecat = torch.tensor(np.concatenate([np.r_[np.asarray(e, dtype=np.float64), 0.0]
                                        for _, _, e in mats]), device=dev)
    opts = mr3.make_opts(abs_split=1, profile=1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        mr3.stemr_batched(n_off, dcat, ecat, opts=opts)
    torch.cuda.synchronize()
    ms = []
    res = None
    for k in range(max(args.steps, 3)):
        flush.fill_(float(k))
        a, b = _events()
        a.record()
        res = mr3.stemr_batched(n_off, dcat, ecat, opts=opts)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    _, w, Z, z_off, info = res
    acc = []
    for b, (kind, d, e) in enumerate(mats):
        n = sizes[b]
        wb = w[n_off[b]:n_off[b] + n]
        Zb = Z[z_off[b]:z_off[b] + n * n].view(n, n).t()
        tn = max(abs(float(wb[0])), abs(float(wb[-1])))
        r, o = gpu_gates(dcat[n_off[b]:n_off[b] + n], ecat[n_off[b]:n_off[b] + n], wb, Zb, tn)
        acc.append({"matrix": kind, "n": n, "resid": round(r, 4), "orth": round(o, 4)})
    med = statistics.median(ms)
    return {"metric": "eigenpairs/s (n=8192 all, FP64) with opts.abs_split",
            "value": sum(sizes) / (med / 1e3), "unit": "eigenpairs/s", "ms_per_step": med,
            "ms_all": ms, "accuracy": acc, "status": info["status"],
            "untested_rrr": info["untested_rrr"], "new_rrr": info["new_rrr"],
            "dmax": info["dmax"], "largest_cluster": info["largest_cluster"],
            "kernel_ms": [round(x, 3) for x in info["kernel_ms"]],
            "note": "opt-in: pieces cut out by absolute gaps are shifted inside the root's "
                    "spectrum; representations failing the growth test are accepted by least "
                    "growth (status 1), so the 10 n eps orthogonality is not guaranteed"}


def backward_leg(args):
    """Backward vs forward at n = 4096 (uniform(-1,1) d and e seeds 501, 502, all
    eigenpairs): loss sum(g . lambda) + sum(G o Z), g and G standard normal (seeds 503,
    504); median device times of mr3_stemr and of mr3_backward."""
    import torch
    import paper_1401_4950_gb300 as mr3
    dev = torch.device("cuda", torch.cuda.current_device())
    n = args.n_bwd
    d, e = tm.random_uniform(n, 501, 502)
    g = torch.tensor(tm.normal(503, n), device=dev)
    G = torch.tensor(tm.normal(504, n * n).reshape(n, n), device=dev).t().contiguous().t()
    dt, et = torch.tensor(d, device=dev), torch.tensor(e, device=dev)
    for _ in range(2):
        w, Z, _ = mr3.stemr(dt, et)
        mr3.backward(w, Z, g, G)
    torch.cuda.synchronize()
    reps = max(5, min(args.steps, 10))
    tf, tb = [], []
    for _ in range(reps):
        a, b = _events()
        a.record()
        w, Z, _ = mr3.stemr(dt, et)
        b.record()
        c, dd_ = _events()
        c.record()
        mr3.backward(w, Z, g, G)
        dd_.record()
        torch.cuda.synchronize()
        tf.append(a.elapsed_time(b))
        tb.append(c.elapsed_time(dd_))
    wc = w.cpu().numpy()
    fm, bm = statistics.median(tf), statistics.median(tb)
    # the per-eigenpair adjoint (mr3_backward_solve) on the same problem, and on the middle
    # 20% of the eigenpairs (a subset, which the dense path does not take)
    ts = []
    for _ in range(reps):
        a, b = _events()
        a.record()
        mr3.backward_solve(dt, et, w, Z, g, G)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    il, iu = 2 * n // 5 + 1, 3 * n // 5
    ws, Zs, _ = mr3.stemr(dt, et, rng="I", il=il, iu=iu)
    gs, Gs = g[il - 1:iu].contiguous(), G[:, il - 1:iu]
    tsub = []
    for _ in range(reps):
        a, b = _events()
        a.record()
        mr3.backward_solve(dt, et, ws, Zs, gs, Gs)
        b.record()
        torch.cuda.synchronize()
        tsub.append(a.elapsed_time(b))
    sm, ssub = statistics.median(ts), statistics.median(tsub)
    return {"metric": "backward / forward time (n=%d, all eigenpairs, FP64)" % n,
            "value": bm / fm, "unit": "ratio", "forward_ms": fm, "backward_ms": bm,
            "backward_path": "dense: two n^3 products as exact sums of bf16 slice products "
                             "on the library's tcgen05 kernel",
            "solve_backward_ms": sm, "solve_over_forward": sm / fm,
            "subset": {"il": il, "iu": iu, "solve_backward_ms": ssub},
            "min_eigenvalue_gap": float(np.min(np.diff(wc))) if n > 1 else None}


def subset_leg(args):
    """Subset workload: eigenpairs 8001..12000 of the n = 20000 glued Wilkinson matrix (W21+
    blocks glued by 1e-8), binary64 tree vs double-double tree, with the scaled residual and
    orthogonality of each result."""
    import torch
    import paper_1401_4950_gb300 as mr3
    dev = torch.device("cuda", torch.cuda.current_device())
    n, il, iu = 20000, 8001, 12000
    d, e = tm.make("glued_wilkinson", n)
    dt, et = torch.tensor(d, device=dev), torch.tensor(e, device=dev)
    w1, _, _ = mr3.stemr(dt, et, rng="I", il=1, iu=1)
    wn, _, _ = mr3.stemr(dt, et, rng="I", il=n, iu=n)
    tnorm = max(abs(w1.item()), abs(wn.item()))
    out = {"metric": "eigenpairs/s (n=20000 glued Wilkinson, eigenpairs 8001..12000)",
           "unit": "eigenpairs/s", "config": "MRRR subset, n=20000 glued W21+ (e=1e-8 at "
                                             "joins), il=8001, iu=12000"}
    for name, prec in (("fp64", mr3.FP64), ("dd", mr3.DD)):
        opts = mr3.make_opts(prec=prec, profile=1)
        for _ in range(2):
            mr3.stemr(dt, et, rng="I", il=il, iu=iu, opts=opts)
        torch.cuda.synchronize()
        reps = max(3, min(args.steps, 5))
        a, b = _events()
        a.record()
        for _ in range(reps):
            w, Z, info = mr3.stemr(dt, et, rng="I", il=il, iu=iu, opts=opts)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / reps
        resid, orth = gpu_gates(dt, et, w, Z, tnorm)
        out[name] = {"value": (iu - il + 1) / (ms * 1e-3), "ms": ms, "resid": round(resid, 4),
                     "orth": round(orth, 4), "dmax": info["dmax"],
                     "nclusters": info["nclusters"], "largest_cluster": info["largest_cluster"],
                     "rqi_iters": info["rqi_iters"], "bisect_fallbacks": info["bisect_fallbacks"],
                     "status": info["status"],
                     "kernel_ms": [round(x, 3) for x in info["kernel_ms"]]}
        del w, Z
    return out


def left_subset_leg(args):
    """Ch. 4 subset experiment: eigenpairs 1..iu at the left end of the spectrum of order
    10,001 matrices (1-2-1, Wilkinson, uniform(-1,1)), time against the fraction iu / n.
    MRRR's cost is proportional to the number of eigenpairs computed; reported as the
    median device time per fraction and its ratio to the time for all eigenpairs."""
    import torch
    import paper_1401_4950_gb300 as mr3
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 10001
    fracs = (0.01, 0.1, 0.25, 0.5, 1.0)
    out = {"metric": "left-end subset time against the fraction of eigenpairs (n=10001)",
           "unit": "ms", "fractions": list(fracs)}
    for kind, seeds in (("one_two_one", None), ("wilkinson", None), ("random", (601, 602))):
        d, e = tm.random_uniform(n, *seeds) if seeds else tm.make(kind, n)
        dt, et = torch.tensor(d, device=dev), torch.tensor(e, device=dev)
        times = []
        for f in fracs:
            iu = max(1, int(round(f * n)))
            for _ in range(2):
                mr3.stemr(dt, et, rng="I", il=1, iu=iu)
            tt = []
            for _ in range(3):
                a, b = _events()
                a.record()
                w, Z, _ = mr3.stemr(dt, et, rng="I", il=1, iu=iu)
                b.record()
                torch.cuda.synchronize()
                tt.append(a.elapsed_time(b))
                del w, Z
            times.append(statistics.median(tt))
        out[kind] = {"ms": [round(t, 3) for t in times],
                     "relative_to_all": [round(t / times[-1], 4) for t in times]}
    return out


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
    ap.add_argument("--no-extras", action="store_true",
                    help="headline step only (no batched, backward and subset legs)")
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--n-bwd", type=int, default=4096)
    ap.add_argument("--solver", default="batched", choices=["batched", "single"],
                    help="the step's matrices in one mr3_stemr_batched call, or one mr3_stemr "
                         "call each")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "dd"],
                    help="representation tree in binary64 or double-double (Ch. 5)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's launch-shape rules instead of tuning the RQI "
                         "team size and bisection warps per SM on the workload first")
    ap.add_argument("--no-per-matrix", action="store_true",
                    help="batched leg: skip the one-call-per-matrix comparison (profiling)")
    ap.add_argument("--abs-split", action="store_true",
                    help="amend the root classification by absolute gaps (opts.abs_split)")
    ap.add_argument("--erep", action="store_true",
                    help="binary64 child representations as e-representations (opts.erep)")
    ap.add_argument("--leg", default=None,
                    choices=["batched", "backward", "subset", "left_subsets"],
                    help="print only one of the extra legs as its own JSON line")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, args.config, rank)
        return
    if args.leg:
        import torch
        torch.cuda.set_device(0)
        leg = {"batched": batched_leg, "backward": backward_leg, "subset": subset_leg,
               "left_subsets": left_subset_leg}[args.leg]
        print(json.dumps(leg(args)), flush=True)
        return
    run_gpu(args, args.config, rank, world)


if __name__ == "__main__":
    main()
