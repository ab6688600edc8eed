"""The mixed-precision variant (opts.prec = DD: the representation tree in double-double,
gaptol 1e-10) against the CPU oracle, and its structural effect on the tree (Ch. 5)."""
import numpy as np
import pytest

import testmats as tm
from _checks import check_eigenpairs
from oracle import metrics as M

pytestmark = pytest.mark.gpu


def _solve(d, e, prec, **kw):
    import torch
    import paper_1401_4950_gb300 as mr3
    dt = torch.tensor(np.asarray(d, dtype=np.float64), device="cuda")
    et = torch.tensor(np.asarray(e, dtype=np.float64) if len(e) else np.zeros(1), device="cuda")
    w, Z, info = mr3.stemr(dt, et, opts=mr3.make_opts(prec=prec), **kw)
    torch.cuda.synchronize()
    return w.cpu().numpy(), Z.cpu().numpy(), info


CASES = [("random", 1), ("random", 2), ("random", 37), ("random", 1000), ("one_two_one", 1000),
         ("wilkinson", 21), ("wilkinson", 1001), ("glued_wilkinson", 42),
         ("glued_wilkinson", 1000), ("clement", 501), ("legendre", 300), ("laguerre", 300),
         ("hermite", 400), ("uniform_eigs", 300), ("geometric_eigs", 1000)]


@pytest.mark.parametrize("kind,n", CASES)
def test_dd_matches_oracle(cuda, kind, n):
    import paper_1401_4950_gb300 as mr3
    d, e = tm.make(kind, n, seed=301)
    w, Z, info = _solve(d, e, mr3.DD)
    assert info["m"] == n
    # every family, the tight-pair ones included, within the 10 n eps gates
    check_eigenpairs(d, e, w, Z)
    # the Rayleigh-quotient iteration converges from the bisection's intervals: a fallback
    # to bisection is the exception (its intervals must bracket the double-double
    # representation's eigenvalues)
    assert info["bisect_fallbacks"] <= max(1, n // 100), info["bisect_fallbacks"]


@pytest.mark.parametrize("kind,n", [("wilkinson", 1001), ("glued_wilkinson", 1000),
                                    ("random", 1000), ("one_two_one", 1000)])
def test_dd_orthogonality_beats_fp64_tree(cuda, kind, n):
    # Ch. 5: with the tree in double-double the orthogonality is no longer limited by
    # k n eps_x / gaptol; the binary64 tree's level on these families is the reference
    import paper_1401_4950_gb300 as mr3
    d, e = tm.make(kind, n, seed=302)
    _, Z64, _ = _solve(d, e, mr3.FP64)
    _, Zdd, _ = _solve(d, e, mr3.DD)
    o64, odd = M.scaled_orthogonality(Z64), M.scaled_orthogonality(Zdd)
    assert odd <= 1.0, (odd, o64)
    assert odd <= o64 + 0.05, (odd, o64)


def test_dd_tree_is_shallow(cuda):
    # glued Wilkinson W21+ blocks: the 1e-8 glue leaves clusters of eigenvalues within
    # ~1e-8 of each other; at gaptol 1e-10 one shift separates them (d_max <= 2, Ch. 5)
    import paper_1401_4950_gb300 as mr3
    d, e = tm.make("glued_wilkinson", 2100, seed=303)
    _, _, i64 = _solve(d, e, mr3.FP64)
    w, Z, idd = _solve(d, e, mr3.DD)
    assert idd["dmax"] <= 2, idd
    assert idd["dmax"] <= i64["dmax"]
    check_eigenpairs(d, e, w, Z, vec_compare=False)


@pytest.mark.parametrize("il,iu", [(1, 1), (40, 60), (190, 200)])
def test_dd_index_subsets(cuda, il, iu):
    import paper_1401_4950_gb300 as mr3
    d, e = tm.make("glued_wilkinson", 210, seed=304)
    w, Z, info = _solve(d, e, mr3.DD, rng="I", il=il, iu=iu)
    assert info["m"] == iu - il + 1
    check_eigenpairs(d, e, w, Z, il=il, iu=iu)


def test_dd_rqi_fallback(cuda):
    # forced non-convergence: every singleton is finished by double-double bisection
    import torch
    import paper_1401_4950_gb300 as mr3
    d, e = tm.make("random", 300, seed=305)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    w, Z, info = mr3.stemr(dt, et, opts=mr3.make_opts(prec=mr3.DD, fault_mask=mr3.FAULT_RQI_NOCONV))
    torch.cuda.synchronize()
    assert info["bisect_fallbacks"] == info["m"]
    check_eigenpairs(d, e, w.cpu().numpy(), Z.cpu().numpy())


def test_dd_batched(cuda):
    import torch
    import paper_1401_4950_gb300 as mr3
    sizes = [1, 5, 64, 300, 17]
    mats = [tm.make("random", n, seed=310 + k) for k, n in enumerate(sizes)]
    n_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    dcat = np.concatenate([np.asarray(m[0], dtype=np.float64) for m in mats])
    ecat = np.concatenate([np.r_[np.asarray(m[1], dtype=np.float64), 0.0] for m in mats])
    m, w, Z, z_off, info = mr3.stemr_batched(n_off, torch.tensor(dcat, device="cuda"),
                                             torch.tensor(ecat, device="cuda"),
                                             opts=mr3.make_opts(prec=mr3.DD))
    torch.cuda.synchronize()
    w, Z = w.cpu().numpy(), Z.cpu().numpy()
    for b, (d, e) in enumerate(mats):
        n, k = sizes[b], int(m[b])
        assert k == n
        wb = w[n_off[b]:n_off[b] + k]
        Zb = Z[z_off[b]:z_off[b] + n * k].reshape(k, n).T
        check_eigenpairs(d, e, wb, Zb)
