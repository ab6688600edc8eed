"""Seeded synthetic tridiagonal test matrices.

This module only produces input arrays (diagonal ``d`` and off-diagonal ``e``
of a real symmetric tridiagonal T, plus seeded right-hand data for the
backward pass).  It contains none of the eigensolver's arithmetic, so both the
CPU oracle and the CUDA path may consume its output.

Random numbers come from a counter-based generator: SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), applied
to ``seed + (i + 1) * 0x9E3779B97F4A7C15`` for element index ``i``.  The top 53
bits of the mixed word give a uniform double in [0, 1).

Matrix families follow the thesis' test-matrix appendix (App. D) and the
workloads it measures:
  * 1-2-1        -- d = 2, e = -1; eigenvalues 2 - 2 cos(pi k/(n+1)) (App. D)
  * Wilkinson    -- d = |i - (n-1)/2| (0-based i), e = 1 (App. D; even n allowed,
                    which gives the half-integer diagonal n/2-1/2 ... 1/2 ... n/2-1/2)
  * glued Wilkinson -- W21+ blocks (d = |j - 10|, j = i mod 21) with e = 1 inside a
                    block and a small glue value between blocks (ref. "glued" in Ch. 3)
  * Clement, Legendre, Laguerre, Hermite (App. D)
  * Uniform and Geometric (App. D) -- tridiagonals with a prescribed spectrum
                    lambda_k = eps + (k-1)(1-eps)/(n-1) and lambda_k = eps^((n-k)/(n-1)),
                    eps = 2^-53, built by Lanczos with full reorthogonalisation on
                    diag(lambda) from a seeded random start vector
  * uniform random -- d_i, e_i i.i.d. uniform(-1, 1)
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """SplitMix64 outputs for counters start..start+count-1 of stream ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(seed: int, count: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, count)


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]            # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


# ---------------------------------------------------------------- matrix families

def random_uniform(n: int, seed_d: int, seed_e: int):
    return uniform(seed_d, n), uniform(seed_e, max(n - 1, 0))


def one_two_one(n: int):
    return np.full(n, 2.0), np.full(max(n - 1, 0), -1.0)


def wilkinson(n: int):
    i = np.arange(n, dtype=np.float64)
    return np.abs(i - (n - 1) / 2.0), np.ones(max(n - 1, 0))


def glued_wilkinson(n: int, block: int = 21, glue: float = 1e-8):
    """W(block)+ blocks repeated to length n (last block truncated), glued by ``glue``."""
    i = np.arange(n)
    j = i % block
    m = (block - 1) / 2.0
    d = np.abs(j - m).astype(np.float64)
    e = np.ones(max(n - 1, 0))
    joins = np.arange(block - 1, n - 1, block)     # e between rows block-1 and block, ...
    e[joins] = glue
    return d, e


def clement(n: int):
    k = np.arange(1, n, dtype=np.float64)
    return np.zeros(n), np.sqrt(k * (n - k))


def legendre(n: int):
    k = np.arange(2, n + 1, dtype=np.float64)
    return np.zeros(n), k / np.sqrt((2 * k - 1) * (2 * k + 1))


def laguerre(n: int):
    d = 2.0 * np.arange(1, n + 1, dtype=np.float64) + 1.0
    e = np.arange(2, n + 1, dtype=np.float64)
    return d, e


def hermite(n: int):
    return np.zeros(n), np.sqrt(np.arange(1, n, dtype=np.float64))


UNIT_ROUNDOFF = 2.0 ** -53


def uniform_spectrum(n: int) -> np.ndarray:
    """App. D, Uniform: lambda_k = eps + (k-1)(1-eps)/(n-1), k = 1..n."""
    if n == 1:
        return np.array([UNIT_ROUNDOFF])
    k = np.arange(1, n + 1, dtype=np.float64)
    return UNIT_ROUNDOFF + (k - 1) * (1.0 - UNIT_ROUNDOFF) / (n - 1)


def geometric_spectrum(n: int) -> np.ndarray:
    """App. D, Geometric: lambda_k = eps^((n-k)/(n-1)), k = 1..n."""
    if n == 1:
        return np.array([1.0])
    k = np.arange(1, n + 1, dtype=np.float64)
    return UNIT_ROUNDOFF ** ((n - k) / (n - 1))


def lanczos_tridiagonal(lam, seed: int = 7001, device=None):
    """A symmetric tridiagonal T = Q^T diag(lam) Q with the eigenvalues lam (up to rounding):
    n steps of Lanczos on diag(lam) from a seeded normal start vector, with full
    reorthogonalisation (classical Gram-Schmidt applied twice) against every earlier
    Lanczos vector.  Returns (d, e).  With `device` (a torch device) the vectors live
    there; the output is a numpy array either way."""
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.shape[0]
    if device is None:
        xp_lam = lam
        Q = np.zeros((n, n))
        q = normal(seed, n)
        dot = np.dot

        def mv(A, x):
            return A @ x
    else:
        import torch
        xp_lam = torch.tensor(lam, device=device)
        Q = torch.zeros((n, n), dtype=torch.float64, device=device)
        q = torch.tensor(normal(seed, n), device=device)
        dot = torch.dot

        def mv(A, x):
            return A @ x
    q = q / float(dot(q, q)) ** 0.5
    d = np.zeros(n)
    e = np.zeros(max(n - 1, 0))
    for j in range(n):
        Q[j] = q
        w = xp_lam * q
        d[j] = float(dot(q, w))
        for _ in range(2):  # full reorthogonalisation, twice
            w = w - mv(Q[: j + 1].T, mv(Q[: j + 1], w))
        if j == n - 1:
            break
        b = float(dot(w, w)) ** 0.5
        e[j] = b
        if b == 0.0:  # invariant subspace (cannot happen with distinct lam and a generic start)
            raise ValueError("Lanczos breakdown at step %d" % j)
        q = w / b
    return d, e


def uniform_eigs(n: int, seed: int = 7001, device=None):
    return lanczos_tridiagonal(uniform_spectrum(n), seed, device)


def geometric_eigs(n: int, seed: int = 7002, device=None):
    return lanczos_tridiagonal(geometric_spectrum(n), seed, device)


FAMILIES = {
    "one_two_one": one_two_one,
    "wilkinson": wilkinson,
    "glued_wilkinson": glued_wilkinson,
    "clement": clement,
    "legendre": legendre,
    "laguerre": laguerre,
    "hermite": hermite,
    "uniform_eigs": uniform_eigs,
    "geometric_eigs": geometric_eigs,
}


def make(kind: str, n: int, seed: int = 0):
    """Build a test matrix by family name; ``random`` uses seeds (seed, seed + 1)."""
    if kind == "random":
        return random_uniform(n, seed, seed + 1)
    return FAMILIES[kind](n)


# ---------------------------------------------------------------- batched workload

def batched_sizes(nb: int, seed: int, nmin: int = 32, nmax: int = 1024) -> np.ndarray:
    """Sizes n_b = nmin + floor(u * (nmax - nmin + 1)), u uniform in [0, 1)."""
    u = uniform01(seed, nb)
    return (nmin + np.floor(u * (nmax - nmin + 1))).astype(np.int64)


def batched_random(nb: int, size_seed: int = 401, d_seed0: int = 402, e_seed0: int = 403,
                   nmin: int = 32, nmax: int = 1024):
    """Packed batch of uniform(-1,1) tridiagonals.

    Returns (sizes, n_off, d, e, e_off) where matrix b occupies d[n_off[b]:n_off[b+1]] and
    e[n_off[b]:n_off[b+1]-1] (e is packed with the same offsets as d; its last slot of each
    matrix is unused and set to 0).
    """
    sizes = batched_sizes(nb, size_seed, nmin, nmax)
    n_off = np.zeros(nb + 1, dtype=np.int64)
    n_off[1:] = np.cumsum(sizes)
    d = np.empty(n_off[-1])
    e = np.zeros(n_off[-1])
    for b in range(nb):
        nbk = int(sizes[b])
        d[n_off[b]:n_off[b + 1]] = uniform(d_seed0 + 2 * b, nbk)
        e[n_off[b]:n_off[b + 1] - 1] = uniform(e_seed0 + 2 * b, nbk - 1)
    return sizes, n_off, d, e
