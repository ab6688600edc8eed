"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms printed in the thesis (App. D), brute-force Jacobi, trace identities,
Sturm-count consistency, and an independent library eigensolver (LAPACK via numpy)."""
import numpy as np
import pytest

import oracle
import testmats as tm
from oracle import metrics as M

EPS = oracle.EPS


def _closed_121(n):
    k = np.arange(1, n + 1)
    return 2.0 - 2.0 * np.cos(np.pi * k / (n + 1))


@pytest.mark.parametrize("n", [1, 2, 3, 10, 100, 257, 1000])
def test_121_eigenvalues_closed_form(n):
    # App. D: the 1-2-1 matrix has eigenvalues 2 - 2 cos(pi k / (n+1)).
    d, e = tm.one_two_one(n)
    w = oracle.eigvals(d, e)
    assert np.max(np.abs(w - _closed_121(n))) <= 8 * EPS * 4


@pytest.mark.parametrize("n", [5, 60, 200])
def test_121_eigenvectors_closed_form(n):
    # Textbook: z_k(j) = sqrt(2/(n+1)) sin(j k pi / (n+1)).  One long absolute-gap chain,
    # so this also exercises the re-orthogonalisation.
    d, e = tm.one_two_one(n)
    w = oracle.eigvals(d, e)
    Z = oracle.eigvecs(d, e, w)
    j = np.arange(1, n + 1)[:, None]
    k = np.arange(1, n + 1)[None, :]
    Zx = np.sqrt(2.0 / (n + 1)) * np.sin(j * k * np.pi / (n + 1))
    Zx = M.align_signs(Z, Zx)
    gaps = np.diff(_closed_121(n)).min()
    assert np.max(np.abs(Z - Zx)) <= 200 * n * EPS * 4 / gaps


@pytest.mark.parametrize("n", [2, 7, 30, 64])
def test_jacobi_reproduces_121_closed_form(n):
    d, e = tm.one_two_one(n)
    w, V = oracle.jacobi(oracle.dense(d, e))
    assert np.max(np.abs(w - _closed_121(n))) <= 50 * n * EPS * 4
    assert np.max(np.abs(V.T @ V - np.eye(n))) <= 50 * n * EPS


@pytest.mark.parametrize("n", [2, 3, 10, 11, 64])
def test_clement_integer_spectrum(n):
    # App. D (Clement): beta_k = sqrt(k (n-k)); read as eigenvalues -(n-1), -(n-3), ..., n-1.
    d, e = tm.clement(n)
    w = oracle.eigvals(d, e)
    expect = np.arange(-(n - 1), n, 2, dtype=np.float64)
    assert np.max(np.abs(w - expect)) <= 16 * n * EPS * n
    wj, _ = oracle.jacobi(oracle.dense(d, e))
    assert np.max(np.abs(wj - expect)) <= 100 * n * EPS * n


def _jacobi_vs_bisection(d, e, tol_scale=100):
    n = len(d)
    wj, V = oracle.jacobi(oracle.dense(d, e))
    w = oracle.eigvals(d, e)
    tn = max(abs(w[0]), abs(w[-1]), 1e-300)
    assert np.max(np.abs(w - wj)) <= tol_scale * n * EPS * tn
    return w, wj, V


@pytest.mark.parametrize("kind,n", [("random", 1), ("random", 2), ("random", 17), ("random", 64),
                                    ("wilkinson", 21), ("wilkinson", 64), ("glued_wilkinson", 42),
                                    ("legendre", 40), ("laguerre", 30), ("hermite", 50),
                                    ("clement", 33)])
def test_bisection_matches_jacobi(kind, n):
    d, e = tm.make(kind, n, seed=7)
    _jacobi_vs_bisection(d, e)


@pytest.mark.parametrize("kind,n", [("random", 64), ("wilkinson", 21), ("glued_wilkinson", 42),
                                    ("hermite", 40)])
def test_inverse_iteration_matches_jacobi_vectors(kind, n):
    d, e = tm.make(kind, n, seed=3)
    w, wj, V = _jacobi_vs_bisection(d, e)
    Z = oracle.eigvecs(d, e, w)
    tn = max(abs(w[0]), abs(w[-1]))
    assert M.scaled_residual(d, e, w, Z, tn) <= 10
    assert M.scaled_orthogonality(Z) <= 10
    # compare only well-separated vectors (unique up to sign)
    g = np.full(n, np.inf)
    g[1:] = np.minimum(g[1:], np.diff(wj))
    g[:-1] = np.minimum(g[:-1], np.diff(wj))
    sep = g > 1e-6 * tn
    Za = M.align_signs(V, Z)
    err = np.abs(Za - V).max(axis=0)
    assert np.all(err[sep] <= 1e3 * n * EPS * tn / g[sep])


def test_wilkinson_near_pairs():
    # App. D: almost all eigenvalues of Wilkinson matrices come in increasingly close pairs.
    d, e = tm.wilkinson(21)
    w = oracle.eigvals(d, e)
    top_gaps = w[-1::-2][:5] - w[-2::-2][:5]
    assert np.all(top_gaps[:-1] < top_gaps[1:])  # gaps shrink toward the top
    assert top_gaps[0] < 1e-12


@pytest.mark.parametrize("kind,n", [("random", 500), ("one_two_one", 300), ("wilkinson", 301),
                                    ("glued_wilkinson", 420), ("laguerre", 200)])
def test_trace_identities(kind, n):
    # sum lambda = trace T ; sum lambda^2 = ||T||_F^2 = sum d^2 + 2 sum e^2
    d, e = tm.make(kind, n, seed=11)
    w = oracle.eigvals(d, e)
    tn = max(abs(w[0]), abs(w[-1]))
    assert abs(w.sum() - d.sum()) <= 4 * n * n * EPS * tn
    fro2 = (d * d).sum() + 2.0 * (e * e).sum()
    assert abs((w * w).sum() - fro2) <= 8 * n * n * EPS * tn * tn


@pytest.mark.parametrize("kind,n", [("random", 400), ("wilkinson", 101), ("one_two_one", 256)])
def test_sturm_counts_between_eigenvalues(kind, n):
    d, e = tm.make(kind, n, seed=5)
    w = oracle.eigvals(d, e)
    mids = 0.5 * (w[:-1] + w[1:])
    ok = np.diff(w) > 1e-9 * max(abs(w[0]), abs(w[-1]))
    for k, x in enumerate(mids):
        if ok[k]:
            assert oracle.negcount(d, e, x) == k + 1
    assert oracle.negcount(d, e, w[0] - 1.0) == 0
    assert oracle.negcount(d, e, w[-1] + 1.0) == n


@pytest.mark.parametrize("scale", [1.0, 1e-30, 1e30])
@pytest.mark.parametrize("n", [60, 61])
def test_sturm_count_at_an_exactly_zero_pivot(n, scale):
    # T = s (I + 1e-12 J): at sigma = s the first pivot is exactly zero.  The spectrum
    # s (1 + 2e-12 cos(k pi / (n + 1))) is symmetric about s; for odd n, s itself is the
    # middle eigenvalue.  The count of eigenvalues strictly below s is floor(n / 2) either
    # way; just above s (closer than the nearest eigenvalue s (1 + ~5e-14)) it is
    # ceil(n / 2).
    d, e = np.full(n, scale), np.full(n - 1, 1e-12 * scale)
    assert oracle.negcount(d, e, scale) == n // 2
    assert oracle.negcount(d, e, scale * (1.0 + 1e-14)) == n - n // 2
    w = oracle.eigvals(d, e)
    k = np.arange(1, n + 1)
    wt = np.sort(scale * (1.0 + 2e-12 * np.cos(np.pi * k / (n + 1))))
    assert np.max(np.abs(w - wt)) <= 4 * n * EPS * scale


@pytest.mark.parametrize("kind,n", [("random", 300), ("glued_wilkinson", 210)])
def test_against_lapack(kind, n):
    # numpy.linalg.eigvalsh (LAPACK, a different algorithm) as an outside reference.
    d, e = tm.make(kind, n, seed=9)
    w = oracle.eigvals(d, e)
    wl = np.linalg.eigvalsh(oracle.dense(d, e))
    tn = max(abs(wl[0]), abs(wl[-1]))
    assert np.max(np.abs(w - wl)) <= 4 * n * EPS * tn


def test_gershgorin_contains_spectrum_and_abs_beta1():
    # G6 reading: |beta_1| in the first row; a negative beta_1 must not shrink the interval.
    d = np.array([0.0, 0.0, 0.0])
    e = np.array([-1.0, 0.5])
    gl, gu = oracle.gershgorin(d, e)
    w = oracle.eigvals(d, e)
    assert gl <= w[0] and w[-1] <= gu
    assert gl <= -1.0 and gu >= 1.0
    # first row decides the lower bound here: beta_1 < 0 must widen, not shrink
    dg, eg = np.array([0.0, 5.0, 5.0]), np.array([-1.0, 0.1])
    gl, gu = oracle.gershgorin(dg, eg)
    wg = np.linalg.eigvalsh(oracle.dense(dg, eg))
    assert gl <= wg[0] and wg[-1] <= gu


def test_split_matrix_and_zero_offdiagonal():
    d = np.array([3.0, 1.0, 2.0, -1.0])
    e = np.array([0.0, 0.5, 0.0])
    w = oracle.eigvals(d, e)
    sub = np.linalg.eigvalsh(np.array([[1.0, 0.5], [0.5, 2.0]]))
    assert np.allclose(np.sort(w), np.sort(np.r_[3.0, -1.0, sub]), atol=1e-14)


def test_count_le_value_range():
    d, e = tm.clement(9)  # eigenvalues -8, -6, ..., 8
    assert oracle.count_le(d, e, -6.5) == 1
    lo, hi = oracle.index_range(d, e, "V", vl=-6.5, vu=2.5)
    assert (lo, hi) == (2, 6)


@pytest.mark.parametrize("n", [11, 101, 501])
def test_clement_vectors_with_zero_eigenvalue(n):
    # odd Clement matrices have the eigenvalue 0, which bisection resolves to a denormal;
    # the inverse iteration must still return finite, orthonormal eigenvectors
    d, e = tm.clement(n)
    w = oracle.eigvals(d, e)
    Z = oracle.eigvecs(d, e, w)
    assert np.all(np.isfinite(Z))
    assert M.scaled_residual(d, e, w, Z, n - 1.0) <= 10
    assert M.scaled_orthogonality(Z) <= 10


@pytest.mark.parametrize("kind,n", [("uniform_eigs", 9), ("uniform_eigs", 200), ("uniform_eigs", 600),
                                    ("geometric_eigs", 9), ("geometric_eigs", 200),
                                    ("geometric_eigs", 600)])
def test_prescribed_spectra_of_app_d(kind, n):
    # App. D, Uniform and Geometric: T is built by Lanczos (full reorthogonalisation) on
    # diag(lambda) with the printed spectrum, so the spectrum is known in closed form; the
    # oracle's bisection must return it to ~n eps ||T|| (||T|| = 1)
    d, e = tm.make(kind, n)
    lam = tm.uniform_spectrum(n) if kind == "uniform_eigs" else tm.geometric_spectrum(n)
    w = oracle.eigvals(d, e)
    assert np.max(np.abs(w - lam)) <= 4 * n * EPS
    if n <= 64:
        wj, _ = oracle.jacobi(oracle.dense(d, e))
        assert np.max(np.abs(wj - lam)) <= 50 * n * EPS
