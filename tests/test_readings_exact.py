"""Exact-arithmetic pins of the thesis' factorization algorithms and of the division-free
forms the kernels run them in.

The identities are checked in rational arithmetic (fractions.Fraction) on small random
inputs, so each either holds exactly or the test fails; no tolerance is involved.  The
checks are against plain definitions: the product of the computed factors, the inverse of
the shifted matrix, and Sylvester's law of inertia.  The last pin, an inequality, runs in
binary64 against LAPACK's eigenvectors.

* Alg. dstqds (Ch. 3, "Eigenvectors of symmetric tridiagonals"): L+ D+ L+^T = L D L^T - tau I.
* Alg. dqds, same section.  Its printed loop assigns the new pivot to u-(i+1) and carries a
  stray symbol in the breakdown test; the reading used throughout the library is
  omega-(i+1) = p(i+1) + d(i) l(i)^2, u-(i) = d(i) l(i) / omega-(i+1),
  p(i) = (p(i+1) / omega-(i+1)) d(i) - tau, omega-(1) = p(1).  The pin: with that reading,
  U- Omega- U-^T = L D L^T - tau I.
* Alg. Getvec: gamma_k = s(k) + d(k) p(k+1) / omega-(k+1) (k < n), gamma_n = s(n) + d(n),
  i.e. s(k) + p(k) + tau.  The twisted factorization N_k Delta_k N_k^T with the middle
  pivot gamma_k (Ch. 3, "Computing with finite precision arithmetic", representation
  forms) has 1 / gamma_k = e_k^T (L D L^T - tau I)^{-1} e_k, and gamma_k = d+_k + omega-_k -
  (d_k + d_{k-1} l_{k-1}^2 - tau) (the diagonal of the shifted matrix).
* The Sturm counts run dstqds division-free: c_0 = 1, a_1 = -sigma,
  c_i = d_i c_{i-1} + a_i, a_{i+1} = dll_i a_i - sigma c_i, so that d+_i = c_i / c_{i-1};
  the envelope test runs dqds backwards as p_k = N_k / M_k with M_k = N + dll_k M,
  N_k = (d_k - tau) N - tau dll_k M.  Both forms equal the quotient forms exactly, and the
  number of sign changes of c is the number of eigenvalues below sigma.
* The envelope bound of the shift's second test (a reading of Alg. "Shifting the spectrum",
  whose envelope test has no formula in the thesis): the weight of a group of eigenvectors
  at index k is at most Lambda (1/|gamma_k| + 1/g).
"""
from fractions import Fraction as F
import random

import numpy as np
import pytest


def _rand_frac(rng, lo=-9, hi=9, den=7):
    while True:
        v = F(rng.randint(lo * den, hi * den), rng.randint(1, den))
        if v != 0:
            return v


def _ldl(rng, n):
    d = [_rand_frac(rng) for _ in range(n)]
    l = [_rand_frac(rng, -3, 3) for _ in range(n - 1)]
    return d, l


def _tridiag_of_ldl(d, l, tau):
    """L D L^T - tau I as a dense Fraction matrix."""
    n = len(d)
    A = [[F(0)] * n for _ in range(n)]
    for i in range(n):
        A[i][i] = d[i] + (d[i - 1] * l[i - 1] ** 2 if i > 0 else 0) - tau
        if i < n - 1:
            A[i][i + 1] = A[i + 1][i] = d[i] * l[i]
    return A


def _lower_product(dp, lp):
    """L D L^T from pivots dp and multipliers lp (unit lower bidiagonal L)."""
    return _tridiag_of_ldl(dp, lp, F(0))


def _upper_product(om, um):
    """U Omega U^T from pivots om and multipliers um (unit upper bidiagonal U)."""
    n = len(om)
    A = [[F(0)] * n for _ in range(n)]
    for i in range(n):
        A[i][i] = om[i] + (om[i + 1] * um[i] ** 2 if i < n - 1 else 0)
        if i < n - 1:
            A[i][i + 1] = A[i + 1][i] = om[i + 1] * um[i]
    return A


def _dstqds(d, l, tau):
    n = len(d)
    s = [F(0)] * n
    dp = [F(0)] * n
    lp = [F(0)] * (n - 1)
    s[0] = -tau
    for i in range(n - 1):
        dp[i] = s[i] + d[i]
        lp[i] = d[i] * l[i] / dp[i]
        s[i + 1] = (s[i] / dp[i]) * d[i] * l[i] * l[i] - tau
    dp[n - 1] = s[n - 1] + d[n - 1]
    return dp, lp, s


def _dqds_reading(d, l, tau):
    n = len(d)
    p = [F(0)] * n
    om = [F(0)] * n
    um = [F(0)] * (n - 1)
    p[n - 1] = d[n - 1] - tau
    for i in range(n - 2, -1, -1):
        om[i + 1] = p[i + 1] + d[i] * l[i] * l[i]
        um[i] = d[i] * l[i] / om[i + 1]
        p[i] = (p[i + 1] / om[i + 1]) * d[i] - tau
    om[0] = p[0]
    return om, um, p


def _inverse_diagonal(A):
    """Diagonal of A^{-1} by exact Gauss-Jordan elimination."""
    n = len(A)
    M = [row[:] + [F(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [M[i][n + i] for i in range(n)]


def _cases(count=12):
    rng = random.Random(20140120)
    out = []
    while len(out) < count:
        n = rng.randint(2, 8)
        d, l = _ldl(rng, n)
        tau = _rand_frac(rng, -5, 5)
        try:
            dp, lp, s = _dstqds(d, l, tau)
            om, um, p = _dqds_reading(d, l, tau)
        except ZeroDivisionError:
            continue
        if any(v == 0 for v in dp + om):
            continue
        out.append((d, l, tau, dp, lp, s, om, um, p))
    return out


CASES = _cases()


@pytest.mark.parametrize("case", range(len(CASES)))
def test_dstqds_reproduces_the_shifted_matrix(case):
    d, l, tau, dp, lp, s, *_ = CASES[case]
    assert _lower_product(dp, lp) == _tridiag_of_ldl(d, l, tau)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_dqds_reading_reproduces_the_shifted_matrix(case):
    d, l, tau, *_, om, um, p = CASES[case]
    assert _upper_product(om, um) == _tridiag_of_ldl(d, l, tau)


def test_dqds_literal_assignment_does_not_factor():
    # the printed loop, read literally, stores the new pivot into u-(i+1) and leaves
    # omega- unset below the last index: its output is not a factorization of the
    # shifted matrix (the reading above is needed)
    d, l, tau, *_ = CASES[0]
    n = len(d)
    om = [F(0)] * n
    um = [F(0)] * (n - 1)
    p = [F(0)] * n
    p[n - 1] = d[n - 1] - tau
    for i in range(n - 2, -1, -1):
        if i + 1 < n - 1:
            um[i + 1] = p[i + 1] + d[i] * l[i] * l[i]
        den = om[i + 1] if om[i + 1] != 0 else F(1)
        um[i] = d[i] * l[i] / den
        p[i] = (p[i + 1] / den) * d[i] - tau
    om[0] = p[0]
    assert _upper_product(om, um) != _tridiag_of_ldl(d, l, tau)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_twist_pivots_are_the_inverse_diagonal(case):
    d, l, tau, dp, lp, s, om, um, p = CASES[case]
    n = len(d)
    A = _tridiag_of_ldl(d, l, tau)
    inv_diag = _inverse_diagonal(A)
    for k in range(n):
        gamma_getvec = s[n - 1] + d[n - 1] if k == n - 1 else s[k] + d[k] * p[k + 1] / om[k + 1]
        gamma_sp = s[k] + p[k] + tau
        gamma_fernando = dp[k] + om[k] - A[k][k]
        assert gamma_getvec == gamma_sp == gamma_fernando
        assert 1 / gamma_getvec == inv_diag[k]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_homogeneous_forward_recurrence_gives_the_dstqds_pivots(case):
    d, l, tau, dp, *_ = CASES[case]
    n = len(d)
    dll = [d[i] * l[i] ** 2 for i in range(n - 1)]
    a, cp = -tau, F(1)
    for i in range(n):
        c = d[i] * cp + a
        assert c / cp == dp[i]
        if i < n - 1:
            a = dll[i] * a - tau * c
        cp = c


@pytest.mark.parametrize("case", range(len(CASES)))
def test_homogeneous_backward_recurrence_gives_the_dqds_auxiliaries(case):
    d, l, tau, *_, om, um, p = CASES[case]
    n = len(d)
    dll = [d[i] * l[i] ** 2 for i in range(n - 1)]
    N, M = d[n - 1] - tau, F(1)
    assert N / M == p[n - 1]
    for k in range(n - 2, -1, -1):
        Mk = N + dll[k] * M
        N = (d[k] - tau) * N - (tau * dll[k]) * M
        M = Mk
        assert N / M == p[k]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_sign_changes_count_the_eigenvalues_below_sigma(case):
    # Sylvester's law of inertia: the negative pivots of L D L^T - sigma I, read off the
    # homogeneous recurrence as sign changes of c, number the eigenvalues below sigma
    d, l, *_ = CASES[case]
    n = len(d)
    dll = [d[i] * l[i] ** 2 for i in range(n - 1)]
    A = np.array([[float(v) for v in row] for row in _tridiag_of_ldl(d, l, F(0))])
    lam = np.linalg.eigvalsh(A)
    for sigma in [F(int(round(x * 8)) + 1, 8) for x in np.linspace(lam[0] - 1, lam[-1] + 1, 9)]:
        if np.min(np.abs(lam - float(sigma))) < 1e-9:
            continue
        a, cp, cnt = -sigma, F(1), 0
        for i in range(n):
            c = d[i] * cp + a
            if c == 0:
                break
            cnt += int((c < 0) != (cp < 0))
            if i < n - 1:
                a = dll[i] * a - sigma * c
            cp = c
        else:
            assert cnt == int(np.sum(lam < float(sigma)))


def _envelope_case(seed):
    rng = np.random.default_rng(1000 + seed)
    n = 40
    dT = rng.uniform(-1, 1, n)
    eT = rng.uniform(-1, 1, n - 1)
    T = np.diag(dT) + np.diag(eT, 1) + np.diag(eT, -1)
    lam, Z = np.linalg.eigh(T)
    j0 = int(rng.integers(2, n - 12))
    j1 = j0 + int(rng.integers(1, 8))
    if seed % 2 == 0:  # shift left of the group
        tau = lam[j0] - 1e-3 * (lam[j0] - lam[j0 - 1])
        Lam = lam[j1] - tau
    else:  # right of it
        tau = lam[j1] + 1e-3 * (lam[j1 + 1] - lam[j1])
        Lam = tau - lam[j0]
    outside = np.r_[lam[:j0], lam[j1 + 1:]]
    g = np.min(np.abs(outside - tau))
    gamma = 1.0 / np.diag(np.linalg.inv(T - tau * np.eye(n)))
    env2 = np.sum(Z[:, j0:j1 + 1] ** 2, axis=1)
    return env2, gamma, Lam, g


@pytest.mark.parametrize("seed", range(6))
def test_envelope_bound_of_the_shift_test(seed):
    # The envelope bound the shift's second test uses (a reading: the thesis names an
    # envelope test without a formula).  With mu_j = lambda_j - tau,
    # 1/gamma_k = sum_j z_j(k)^2 / mu_j; the group's mu_j share one sign and are at most
    # Lambda in magnitude, the others at least g, so
    # env2(k) = sum_{j in group} z_j(k)^2 <= Lambda (1/|gamma_k| + 1/g).
    env2, gamma, Lam, g = _envelope_case(seed)
    assert np.all(env2 <= Lam * (1.0 / np.abs(gamma) + 1.0 / g) * (1 + 1e-8))


def test_envelope_bound_needs_the_outside_term():
    # a planted mistake: without the outside eigenvalues' term 1/g the bound fails
    violated = 0
    for seed in range(6):
        env2, gamma, Lam, g = _envelope_case(seed)
        violated += int(np.any(env2 > Lam / np.abs(gamma) * (1 + 1e-8)))
    assert violated > 0
