"""The classification and representation options of the tree, against the CPU oracle at
the same 10 n eps gates:

* abs_split (opt-in): the root classification amended by absolute gaps (Sec. 3.2.3,
  Sec. 4.2.1); pieces of a relative cluster separated by at least the block's average gap
  get their own child representations, one-member pieces included;
* erep: binary64 child representations kept as e-representations (d, beta), the
  off-diagonal entries shared with the root (Ch. 3, representation forms).
"""
import numpy as np
import pytest

import testmats as tm
from _checks import check_eigenpairs

pytestmark = pytest.mark.gpu

CASES = [("random", 2), ("random", 37), ("random", 1000), ("one_two_one", 100),
         ("one_two_one", 1000), ("wilkinson", 21), ("wilkinson", 1001),
         ("glued_wilkinson", 42), ("glued_wilkinson", 1000), ("clement", 501),
         ("legendre", 300), ("laguerre", 300), ("hermite", 400), ("hermite", 2000),
         ("uniform_eigs", 1000), ("geometric_eigs", 1000)]

FLAGS = [{"abs_split": 1}, {"erep": 1}, {"abs_split": 1, "erep": 1}]
IDS = ["abs", "erep", "abs+erep"]


def _solve(d, e, prec=0, rng="A", il=1, iu=None, **flags):
    import torch
    import paper_1401_4950_gb300 as mr3
    dt = torch.tensor(np.asarray(d, dtype=np.float64), device="cuda")
    et = torch.tensor(np.asarray(e, dtype=np.float64) if len(e) else np.zeros(1), device="cuda")
    w, Z, info = mr3.stemr(dt, et, rng=rng, il=il, iu=iu,
                           opts=mr3.make_opts(prec=prec, **flags))
    torch.cuda.synchronize()
    return w.cpu().numpy(), Z.cpu().numpy(), info


@pytest.mark.parametrize("flags", FLAGS, ids=IDS)
@pytest.mark.parametrize("kind,n", CASES)
def test_all_eigenpairs_match_oracle(cuda, kind, n, flags):
    d, e = tm.make(kind, n, seed=101)
    w, Z, info = _solve(d, e, **flags)
    assert info["m"] == n and info["status"] in (0, 1)
    check_eigenpairs(d, e, w, Z)


@pytest.mark.parametrize("flags", FLAGS, ids=IDS)
@pytest.mark.parametrize("kind,n,il,iu", [("random", 600, 101, 300), ("one_two_one", 800, 1, 80),
                                          ("hermite", 1200, 500, 700),
                                          ("glued_wilkinson", 630, 200, 420)])
def test_index_range(cuda, kind, n, il, iu, flags):
    d, e = tm.make(kind, n, seed=102)
    w, Z, info = _solve(d, e, rng="I", il=il, iu=iu, **flags)
    assert w.shape == (iu - il + 1,)
    check_eigenpairs(d, e, w, Z, il=il, iu=iu)


@pytest.mark.parametrize("kind,n", [("one_two_one", 1000), ("hermite", 1500), ("random", 800),
                                    ("wilkinson", 201)])
def test_double_double_tree_with_abs_split(cuda, kind, n):
    import paper_1401_4950_gb300 as mr3
    d, e = tm.make(kind, n, seed=103)
    w, Z, info = _solve(d, e, prec=mr3.DD, abs_split=1)
    check_eigenpairs(d, e, w, Z)


@pytest.mark.parametrize("kind,n,shrinks", [("one_two_one", 2000, True), ("hermite", 3000, True),
                                            ("uniform_eigs", 2000, False)])
def test_abs_split_shrinks_the_largest_cluster(cuda, kind, n, shrinks):
    # the amendment only ever adds boundaries at the root: the largest cluster cannot grow.
    # It shrinks where the spacing varies (1-2-1, Hermite); on an equispaced spectrum every
    # gap is the average gap and nothing splits.
    d, e = tm.FAMILIES[kind](n, device="cuda") if kind == "uniform_eigs" else tm.make(kind, n, seed=104)
    _, _, i0 = _solve(d, e)
    _, _, i1 = _solve(d, e, abs_split=1)
    assert i1["largest_cluster"] <= i0["largest_cluster"], (i0, i1)
    if shrinks:
        assert i1["largest_cluster"] < i0["largest_cluster"], (i0, i1)


def test_batched_matches_per_matrix_with_flags(cuda):
    # the lanes per cluster end of the end refinement follow the number of clusters in the
    # launch, so a batch's brackets (and shifts) differ from a lone matrix's in the last
    # bits: the two are compared against the same gates, not bit for bit
    import torch
    import paper_1401_4950_gb300 as mr3
    sizes = [300, 57, 1000, 2, 640]
    kinds = ["random", "wilkinson", "one_two_one", "random", "hermite"]
    mats = [tm.make(k, n, seed=105 + b) for b, (k, n) in enumerate(zip(kinds, sizes))]
    n_off = np.zeros(len(sizes) + 1, dtype=np.int64)
    n_off[1:] = np.cumsum(sizes)
    d = np.concatenate([m[0] for m in mats])
    e = np.concatenate([np.r_[m[1], 0.0] for m in mats])
    o = mr3.make_opts(abs_split=1, erep=1)
    _, w, Z, z_off, _ = mr3.stemr_batched(n_off, torch.tensor(d, device="cuda"),
                                          torch.tensor(e, device="cuda"), opts=o)
    for b, n in enumerate(sizes):
        ws, _, _ = _solve(*mats[b], abs_split=1, erep=1)
        wb = w[n_off[b]:n_off[b] + n].cpu().numpy()
        Zb = Z[z_off[b]:z_off[b] + n * n].view(n, n).t().cpu().numpy()
        tn = max(abs(ws[0]), abs(ws[-1]))
        assert np.max(np.abs(wb - ws)) <= 4 * n * 2.0 ** -53 * tn
        check_eigenpairs(*mats[b], wb, Zb)


def test_abs_split_warns_when_interior_shifts_fail(cuda):
    # T = I + 1e-12 J (near-Toeplitz): every piece the absolute-gap split cuts out needs a
    # shift inside the root's spectrum, where the element growth of L D L^T - tau I exceeds
    # the growth test for every candidate.  The representations are then accepted by least
    # growth (Alg. "Shifting the spectrum": accuracy no longer guaranteed), which the call
    # reports as status 1; the default classification (relative gaps only) shifts the one
    # big cluster outside the spectrum and stays at the gates.
    n = 500
    d, e = np.ones(n), np.full(n - 1, 1e-12)
    w, Z, info = _solve(d, e, abs_split=1)
    assert info["status"] == 1 and info["untested_rrr"] > 0, info
    w, Z, info = _solve(d, e)
    assert info["status"] == 0 and info["untested_rrr"] == 0
    check_eigenpairs(d, e, w, Z, w_ref=np.sort(1.0 + 2e-12 * np.cos(np.pi * np.arange(1, n + 1) / (n + 1))),
                     tn=1.0, vec_compare=False)
