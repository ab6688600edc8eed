"""Degenerate and extreme inputs through the C ABI, against the oracle: matrices that split
completely, repeated eigenvalues, extreme scaling, nearly split off-diagonals, and the
smallest orders, with the binary64 and the double-double tree."""
import numpy as np
import pytest

import oracle
import testmats as tm
from _checks import EPS, check_eigenpairs

pytestmark = pytest.mark.gpu


def _solve(d, e, prec=0, **kw):
    import torch
    import paper_1401_4950_gb300 as mr3
    dt = torch.tensor(np.asarray(d, dtype=np.float64), device="cuda")
    et = torch.tensor(np.asarray(e, dtype=np.float64) if len(e) else np.zeros(1), device="cuda")
    w, Z, info = mr3.stemr(dt, et, opts=mr3.make_opts(prec=prec), **kw)
    torch.cuda.synchronize()
    return w.cpu().numpy(), Z.cpu().numpy(), info


@pytest.mark.parametrize("prec", [0, 1])
def test_zero_matrix(cuda, prec):
    # every off-diagonal is zero: n blocks of order one, all eigenvalues 0
    n = 100
    w, Z, info = _solve(np.zeros(n), np.zeros(n - 1), prec)
    assert info["m"] == n and info["nblocks"] == n
    assert np.all(w == 0.0)
    assert np.allclose(np.abs(Z).sum(axis=0), 1.0) and np.allclose(Z.T @ Z, np.eye(n))


@pytest.mark.parametrize("prec", [0, 1])
def test_diagonal_with_repeats(cuda, prec):
    # a split matrix with repeated eigenvalues: ascending output, a unit vector per column
    d = np.array([3.0, -1.0, 3.0, 2.0, -1.0, 3.0, 0.5, 2.0])
    w, Z, info = _solve(d, np.zeros(len(d) - 1), prec)
    assert np.array_equal(w, np.sort(d))
    assert np.allclose(np.abs(Z).max(axis=0), 1.0) and np.allclose(Z.T @ Z, np.eye(len(d)))
    assert np.allclose((Z * d[:, None]).sum(axis=0), w)


@pytest.mark.parametrize("scale", [1e-150, 1e-30, 1e30, 1e150])
@pytest.mark.parametrize("prec", [0, 1])
def test_extreme_scaling(cuda, scale, prec):
    # eigenpairs scale with T: the same relative accuracy at any magnitude
    d, e = tm.random_uniform(300, 701, 702)
    w, Z, _ = _solve(d * scale, e * scale, prec)
    w1, Z1, _ = _solve(d, e, prec)
    assert np.all(np.isfinite(w)) and np.all(np.isfinite(Z))
    tn = max(abs(w1[0]), abs(w1[-1]))
    assert np.max(np.abs(w / scale - w1)) <= 4 * 300 * EPS * tn
    check_eigenpairs(d * scale, e * scale, w, Z, vec_compare=False)


@pytest.mark.parametrize("prec", [0, 1])
def test_nearly_split(cuda, prec):
    # off-diagonals at and just above the splitting threshold eps sqrt(n) ||T||
    n = 400
    d, e = tm.random_uniform(n, 711, 712)
    e = np.array(e)
    e[[50, 51, 200]] = 1e-17
    e[[120, 300]] = 1e-13
    w, Z, info = _solve(d, e, prec)
    assert info["m"] == n
    check_eigenpairs(d, e, w, Z)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_smallest_orders(cuda, n):
    d, e = tm.random_uniform(n, 721, 722)
    for prec in (0, 1):
        w, Z, info = _solve(d, e, prec)
        assert info["m"] == n
        check_eigenpairs(d, e, w, Z)


def test_two_by_two_degenerate(cuda):
    # [[a, b], [b, a]]: eigenvalues a -+ b, vectors (1, -+1)/sqrt(2)
    a, b = 0.75, 1e-3
    w, Z, _ = _solve(np.array([a, a]), np.array([b]))
    assert np.allclose(w, [a - b, a + b], rtol=0, atol=4 * EPS)
    assert np.allclose(np.abs(Z), np.sqrt(0.5), atol=1e-15)


@pytest.mark.parametrize("scale", [1.0, 1e-30, 1e30])
@pytest.mark.parametrize("n", [500, 501])
@pytest.mark.parametrize("prec", [0, 1])
def test_constant_diagonal_tiny_offdiagonal(cuda, prec, n, scale):
    # d = s, e = 1e-12 s: a spectrum of width 4e-12 s around s, symmetric about it (for odd n
    # the middle eigenvalue is s itself), whose relative gaps ~1e-15 the tree resolves by
    # shifts.  Bisection then meets shifts at which a pivot of the Sturm count is exactly
    # zero, a case that has to be counted as the limit at any scale of the data.
    d, e = np.full(n, scale), np.full(n - 1, 1e-12 * scale)
    w, Z, info = _solve(d, e, prec)
    k = np.arange(1, n + 1)
    wt = np.sort(scale * (1.0 + 2e-12 * np.cos(np.pi * k / (n + 1))))
    assert np.max(np.abs(w - wt)) <= 4 * n * EPS * scale
    check_eigenpairs(d, e, w, Z, w_ref=wt, tn=scale, vec_compare=False)
