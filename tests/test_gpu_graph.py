"""The tree's level loop captured in one CUDA graph (opts.graph): bit-for-bit the results of
the host-driven loop, which reads each level's counters, on single matrices, batches of
mixed families and orders, and index and value ranges."""
import numpy as np
import pytest

import testmats as tm
from _checks import check_eigenpairs

pytestmark = pytest.mark.gpu


def _pack(mats):
    sizes = [len(d) for d, _ in mats]
    n_off = np.zeros(len(sizes) + 1, dtype=np.int64)
    n_off[1:] = np.cumsum(sizes)
    d = np.concatenate([np.asarray(m[0], dtype=np.float64) for m in mats])
    e = np.concatenate([np.r_[np.asarray(m[1], dtype=np.float64), 0.0] for m in mats])
    return sizes, n_off, d, e


def _batched(mats, graph, **kw):
    import torch
    import paper_1401_4950_gb300 as mr3
    sizes, n_off, d, e = _pack(mats)
    m, w, Z, z_off, info = mr3.stemr_batched(n_off, torch.tensor(d, device="cuda"),
                                             torch.tensor(e, device="cuda"),
                                             opts=mr3.make_opts(graph=graph), **kw)
    torch.cuda.synchronize()
    return m.copy(), w.cpu().numpy(), Z.cpu().numpy(), z_off, info


MIXED = [("random", 300), ("wilkinson", 201), ("one_two_one", 500), ("glued_wilkinson", 420),
         ("clement", 101), ("hermite", 700), ("random", 2), ("random", 1), ("laguerre", 64)]


def _mats(spec, seed=300):
    return [tm.make(k, n, seed=seed + i) for i, (k, n) in enumerate(spec)]


def test_graph_equals_host_loop_mixed_batch(cuda):
    mats = _mats(MIXED)
    m0, w0, Z0, z0, i0 = _batched(mats, -1)
    m1, w1, Z1, z1, i1 = _batched(mats, 1)
    assert i0["graph_levels"] == 0 and i1["graph_levels"] >= 2
    assert np.array_equal(m0, m1) and np.array_equal(w0, w1) and np.array_equal(Z0, Z1)
    assert i0["nclusters"] == i1["nclusters"] and i0["dmax"] == i1["dmax"]
    _, n_off, _, _ = _pack(mats)
    for b, (d, e) in enumerate(mats):
        n = len(d)
        Zb = Z1[z1[b]:z1[b] + n * n].reshape(n, n).T
        check_eigenpairs(d, e, w1[n_off[b]:n_off[b] + n], Zb)


def test_graph_is_the_default_for_batches(cuda):
    mats = _mats([("random", 400), ("one_two_one", 300)], seed=310)
    import torch
    import paper_1401_4950_gb300 as mr3
    sizes, n_off, d, e = _pack(mats)
    _, _, _, _, info = mr3.stemr_batched(n_off, torch.tensor(d, device="cuda"),
                                         torch.tensor(e, device="cuda"))
    assert info["graph_levels"] >= 1
    # a single matrix keeps the host-driven loop unless asked
    w, Z, info1 = mr3.stemr(torch.tensor(mats[0][0], device="cuda"),
                            torch.tensor(mats[0][1], device="cuda"))
    assert info1["graph_levels"] == 0


@pytest.mark.parametrize("kind,n", [("random", 1000), ("wilkinson", 1001), ("one_two_one", 2000),
                                    ("glued_wilkinson", 1000), ("uniform_eigs", 1000)])
def test_graph_equals_host_loop_single(cuda, kind, n):
    import torch
    import paper_1401_4950_gb300 as mr3
    d, e = (tm.FAMILIES[kind](n, device="cuda") if kind == "uniform_eigs" else tm.make(kind, n, seed=320))
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    w0, Z0, i0 = mr3.stemr(dt, et, opts=mr3.make_opts(graph=-1))
    w1, Z1, i1 = mr3.stemr(dt, et, opts=mr3.make_opts(graph=1))
    assert i1["graph_levels"] >= 1
    assert torch.equal(w0, w1) and torch.equal(Z0, Z1)


def test_graph_equals_host_loop_ranges(cuda):
    mats = _mats([("random", 300), ("hermite", 500), ("wilkinson", 121)], seed=330)
    il, iu = [10, 200, 1], [120, 320, 121]
    r0 = _batched(mats, -1, rng="I", il=il, iu=iu)
    r1 = _batched(mats, 1, rng="I", il=il, iu=iu)
    assert np.array_equal(r0[0], r1[0]) and np.array_equal(r0[1], r1[1]) and np.array_equal(r0[2], r1[2])
    vl, vu = [-0.5, -3.0, 2.0], [0.5, 3.0, 9.5]
    r0 = _batched(mats, -1, rng="V", vl=vl, vu=vu)
    r1 = _batched(mats, 1, rng="V", vl=vl, vu=vu)
    assert np.array_equal(r0[0], r1[0]) and np.array_equal(r0[1], r1[1]) and np.array_equal(r0[2], r1[2])


def test_graph_not_taken_where_it_does_not_apply(cuda):
    import paper_1401_4950_gb300 as mr3
    import torch
    mats = _mats([("random", 200), ("random", 150)], seed=340)
    sizes, n_off, d, e = _pack(mats)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    for o in (mr3.make_opts(prec=mr3.DD, graph=1), mr3.make_opts(abs_split=1, graph=1),
              mr3.make_opts(max_depth=4, graph=1)):
        _, _, _, _, info = mr3.stemr_batched(n_off, dt, et, opts=o)
        assert info["graph_levels"] == 0


def test_graph_bench_workload_sample(cuda):
    # the batched benchmark's shape: 256 uniform(-1, 1) matrices of orders 32..1024
    import torch
    import paper_1401_4950_gb300 as mr3
    sizes, n_off, d, e = tm.batched_random(256)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    out = []
    for g in (-1, 1):
        m, w, Z, z_off, info = mr3.stemr_batched(n_off, dt, et, opts=mr3.make_opts(graph=g))
        out.append((w, Z, info))
    assert out[1][2]["graph_levels"] >= 2
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
