"""CPU pin of the backward formula the library implements (the thesis has no backward pass;
the reading is the first-order perturbation theory of a symmetric eigendecomposition).

For T = Z diag(lambda) Z^T with distinct eigenvalues, a loss
L = sum_i g_i lambda_i + sum_{r,i} G_ri Z_ri (Z sign-normalised: the largest-magnitude
entry of each column positive, ties to the lowest index) has the gradient

    Tbar = Z (diag(g) + F o (Z^T G)) Z^T,   F_ik = D / (D^2 + delta^2),  D = lambda_k - lambda_i,

(F_kk = 0, delta = n eps ||T|| regularising near-equal eigenvalues), and for the tridiagonal
parameters dbar_j = Tbar_jj and ebar_j = Tbar_j,j+1 + Tbar_j+1,j.  The check is central
finite differences of the loss through LAPACK's eigh, on matrices with well separated
eigenvalues; the formula is written out here independently of the library, and a sign
error in D is shown to fail the same check.
"""
import numpy as np
import pytest

EPS = 2.0 ** -53


def _tri(d, e):
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


def _eigh_signed(d, e):
    lam, Z = np.linalg.eigh(_tri(d, e))
    idx = np.argmax(np.abs(Z), axis=0)  # first index of the largest magnitude
    s = np.sign(Z[idx, np.arange(Z.shape[1])])
    return lam, Z * s


def _loss(d, e, g, G):
    lam, Z = _eigh_signed(d, e)
    return float(g @ lam + np.sum(G * Z))


def _grad(d, e, g, G, sign=1.0):
    n = len(d)
    lam, Z = _eigh_signed(d, e)
    tn = max(abs(lam[0]), abs(lam[-1]))
    delta = n * EPS * tn
    D = sign * (lam[None, :] - lam[:, None])  # D_ik = lambda_k - lambda_i
    F = D / (D * D + delta * delta)
    np.fill_diagonal(F, 0.0)
    Tbar = Z @ (np.diag(g) + F * (Z.T @ G)) @ Z.T
    return np.diag(Tbar).copy(), np.diag(Tbar, 1) + np.diag(Tbar, -1)


def _fd(d, e, g, G, h=1e-6):
    n = len(d)
    dd = np.empty(n)
    de = np.empty(n - 1)
    for j in range(n):
        p, m = d.copy(), d.copy()
        p[j] += h
        m[j] -= h
        dd[j] = (_loss(p, e, g, G) - _loss(m, e, g, G)) / (2 * h)
    for j in range(n - 1):
        p, m = e.copy(), e.copy()
        p[j] += h
        m[j] -= h
        de[j] = (_loss(d, p, g, G) - _loss(d, m, g, G)) / (2 * h)
    return dd, de


def _case(seed, n):
    rng = np.random.default_rng(seed)
    while True:
        d = rng.uniform(-1, 1, n)
        e = rng.uniform(0.2, 1, n - 1) * rng.choice([-1.0, 1.0], n - 1)
        lam = np.linalg.eigvalsh(_tri(d, e))
        if np.min(np.diff(lam)) > 0.05:
            break
    g = rng.normal(size=n)
    G = rng.normal(size=(n, n))
    return d, e, g, G


@pytest.mark.parametrize("seed,n", [(1, 4), (2, 6), (3, 8), (4, 10), (5, 12)])
def test_formula_matches_finite_differences(seed, n):
    d, e, g, G = _case(seed, n)
    gd, ge = _grad(d, e, g, G)
    fd, fe = _fd(d, e, g, G)
    scale = max(np.max(np.abs(fd)), np.max(np.abs(fe)), 1.0)
    assert np.max(np.abs(gd - fd)) <= 1e-6 * scale
    assert np.max(np.abs(ge - fe)) <= 1e-6 * scale


def test_eigenvalue_part_is_the_squared_vector_entries():
    # with G = 0: dbar_j = sum_i g_i z_ij^2 and ebar_j = 2 sum_i g_i z_ij z_i,j+1
    d, e, g, _ = _case(7, 9)
    lam, Z = _eigh_signed(d, e)
    gd, ge = _grad(d, e, g, np.zeros((9, 9)))
    assert np.allclose(gd, (Z ** 2) @ g, atol=1e-13)
    assert np.allclose(ge, 2 * (Z[:-1] * Z[1:]) @ g, atol=1e-13)


def test_sign_error_in_the_eigenvalue_differences_is_caught():
    d, e, g, G = _case(2, 6)
    gd, ge = _grad(d, e, g, G, sign=-1.0)
    fd, fe = _fd(d, e, g, G)
    scale = max(np.max(np.abs(fd)), np.max(np.abs(fe)), 1.0)
    assert max(np.max(np.abs(gd - fd)), np.max(np.abs(ge - fe))) > 1e-3 * scale
