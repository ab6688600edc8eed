"""CPU oracle for the symmetric tridiagonal eigenproblem -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  The product (``paper_1401_4950_gb300``) never
imports it and shares no code with it.

The arithmetic lives in ``mr3_oracle.c`` (plain serial C, FP64, no fast-math,
no FMA contraction).  This module compiles it with gcc on first use and wraps it
with ctypes:

* ``gershgorin``      -- App. B, Alg. "Gershgorin"
* ``negcount``        -- App. B, Alg. "NegCount" on T
* ``eigvals``         -- Sec. 3.2.2, Alg. "Bisection" to full accuracy
* ``eigvecs``         -- Sec. 2.3.1, inverse iteration with MGS in absolute-gap chains
* ``stemr``           -- eigenpairs for an index or value range (eigvals + eigvecs)
* ``jacobi``          -- cyclic Jacobi on the dense matrix (brute force, n <= 64)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mr3_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

EPS = np.finfo(np.float64).eps / 2.0  # unit roundoff 2^-53


def compile_source(src: str, out: str) -> str:
    """Compile an oracle C source into a shared library (gcc, -O2, no contraction)."""
    tmp = out + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (oracle/_build/liboracle.so)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


def _bind(path):
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    dp = P(ctypes.c_double)
    ip = P(ctypes.c_int)
    c_int, c_dbl = ctypes.c_int, ctypes.c_double
    lib.orc_gershgorin.argtypes = [c_int, dp, dp, dp, dp]
    lib.orc_gershgorin.restype = None
    lib.orc_negcount.argtypes = [c_int, dp, dp, c_dbl]
    lib.orc_negcount.restype = c_int
    lib.orc_count_le.argtypes = [c_int, dp, dp, c_dbl]
    lib.orc_count_le.restype = c_int
    lib.orc_bisect.argtypes = [c_int, dp, dp, c_int, c_dbl, c_dbl, dp, dp, c_int]
    lib.orc_bisect.restype = c_int
    lib.orc_eigvals.argtypes = [c_int, dp, dp, c_int, c_int, dp, dp, dp]
    lib.orc_eigvals.restype = None
    lib.orc_inverse_iteration.argtypes = [c_int, dp, dp, c_int, dp, dp, c_int,
                                          ctypes.c_uint64, c_dbl, c_int, dp, ip]
    lib.orc_inverse_iteration.restype = c_int
    lib.orc_jacobi.argtypes = [c_int, dp, dp, dp]
    lib.orc_jacobi.restype = c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def use_library(path):
    """Swap the loaded oracle library for a build of another source (the planted-mistake
    tests use this); returns the previous handle for restore_library()."""
    global _lib
    prev = _load()
    with _lock:
        _lib = _bind(path)
    return prev


def restore_library(handle):
    global _lib
    with _lock:
        _lib = handle


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _prep(d, e):
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = d.shape[0]
    e = np.ascontiguousarray(e, dtype=np.float64)[: max(n - 1, 0)]
    if e.shape[0] < max(n - 1, 0):
        raise ValueError("e must hold n-1 entries")
    if e.shape[0] == 0:
        e = np.zeros(1)
    return n, d, e


def gershgorin(d, e):
    n, d, e = _prep(d, e)
    gl, gu = ctypes.c_double(), ctypes.c_double()
    _load().orc_gershgorin(n, _dp(d), _dp(e), ctypes.byref(gl), ctypes.byref(gu))
    return gl.value, gu.value


def negcount(d, e, sigma: float) -> int:
    n, d, e = _prep(d, e)
    return int(_load().orc_negcount(n, _dp(d), _dp(e), float(sigma)))


def count_le(d, e, x: float) -> int:
    n, d, e = _prep(d, e)
    return int(_load().orc_count_le(n, _dp(d), _dp(e), float(x)))


def bisect(d, e, k: int, lo: float, hi: float, rtol: float, atol: float, maxit: int = 4096):
    n, d, e = _prep(d, e)
    a, b = ctypes.c_double(lo), ctypes.c_double(hi)
    it = _load().orc_bisect(n, _dp(d), _dp(e), int(k), rtol, atol, ctypes.byref(a),
                            ctypes.byref(b), maxit)
    return a.value, b.value, it


def eigvals(d, e, il: int = 1, iu: int | None = None, bounds: bool = False):
    """Eigenvalues il..iu (1-based, ascending) to full accuracy by bisection."""
    n, d, e = _prep(d, e)
    if iu is None:
        iu = n
    m = iu - il + 1
    w = np.empty(max(m, 0))
    lo = np.empty(max(m, 0))
    hi = np.empty(max(m, 0))
    if m > 0:
        _load().orc_eigvals(n, _dp(d), _dp(e), il, iu, _dp(w), _dp(lo), _dp(hi))
    return (w, lo, hi) if bounds else w


def eigvecs(d, e, w, seed: int = 12345, chain_tol: float = 1e-3, maxit: int = 5):
    """Inverse-iteration eigenvectors for ascending eigenvalue approximations w."""
    n, d, e = _prep(d, e)
    w = np.ascontiguousarray(w, dtype=np.float64)
    m = w.shape[0]
    Z = np.zeros((m, n))  # row j = column j of the column-major n x m result
    work = np.empty(5 * n)
    iwork = np.empty(n, dtype=np.int32)
    if m > 0:
        _load().orc_inverse_iteration(
            n, _dp(d), _dp(e), m, _dp(w), _dp(Z), n, ctypes.c_uint64(seed), chain_tol, maxit,
            _dp(work), iwork.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return Z.T.copy()


def index_range(d, e, rng: str, vl=None, vu=None, il=None, iu=None):
    """1-based (il, iu) selected by a range: 'A' all, 'I' indices, 'V' values in (vl, vu]."""
    n = len(d)
    if rng == "A":
        return 1, n
    if rng == "I":
        return int(il), int(iu)
    if rng == "V":
        lo = count_le(d, e, vl) + 1
        hi = count_le(d, e, vu)
        return lo, hi
    raise ValueError(rng)


def stemr(d, e, rng: str = "A", vl=None, vu=None, il=None, iu=None, seed: int = 12345):
    """Oracle eigenpairs (w, Z) for the requested range; Z is n x m, columns unit-norm."""
    a, b = index_range(d, e, rng, vl, vu, il, iu)
    w = eigvals(d, e, a, b) if b >= a else np.empty(0)
    Z = eigvecs(d, e, w, seed=seed) if w.size else np.zeros((len(d), 0))
    return w, Z


def jacobi(A):
    """Brute-force eigen-decomposition of a small dense symmetric matrix."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    n = A.shape[0]
    w = np.empty(n)
    V = np.empty((n, n))
    _load().orc_jacobi(n, _dp(A), _dp(w), _dp(V))
    return w, V


def dense(d, e):
    """Dense symmetric matrix of tridiagonal (d, e)."""
    n = len(d)
    T = np.diag(np.asarray(d, dtype=np.float64))
    if n > 1:
        T += np.diag(np.asarray(e[: n - 1], dtype=np.float64), 1)
        T += np.diag(np.asarray(e[: n - 1], dtype=np.float64), -1)
    return T
