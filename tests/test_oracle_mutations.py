"""Planted mistakes: each test compiles a copy of the oracle with one plausible bug
(a dropped term, a wrong sign, a shifted index, a missing absolute value, a skipped
re-orthogonalisation, a wrong rotation) and checks that the oracle pins reject it.
The mistakes are planted on the CPU, in copies; the committed oracle is untouched."""
import os
import tempfile

import numpy as np
import pytest

import oracle
import testmats as tm
from oracle import metrics as M

SRC = os.path.join(os.path.dirname(oracle.__file__), "mr3_oracle.c")

MUTATIONS = {
    "negcount_beta_not_squared": ("piv = (d[i] - sigma) - (b * b) / piv;",
                                  "piv = (d[i] - sigma) - (b) / piv;"),
    "negcount_wrong_sign": ("piv = (d[i] - sigma) - (b * b) / piv;",
                            "piv = (d[i] - sigma) + (b * b) / piv;"),
    "negcount_shifted_index": ("double b = e[i - 1];\n        if (b == 0.0)\n            piv = d[i] - sigma;",
                               "double b = e[i];\n        if (b == 0.0)\n            piv = d[i] - sigma;"),
    "gershgorin_no_abs": ("lo = d[0] - fabs(e[0]);", "lo = d[0] - e[0];"),
    "invit_no_mgs": ("for (int i = 0; i < n; i++) y[i] -= dot * zp[i];",
                     "for (int i = 0; i < n; i++) y[i] -= 0.0 * dot * zp[i];"),
    "jacobi_rotation_sign": ("A[k * n + p] = c * akp - s * akq;", "A[k * n + p] = c * akp + s * akq;"),
    "bisect_wrong_branch": ("if (orc_negcount(n, d, e, w) < k)", "if (orc_negcount(n, d, e, w) <= k)"),
}


def _pins():
    """A compact subset of the pins (closed forms, Jacobi cross-check, LAPACK, vectors)."""
    # 1-2-1 closed form
    n = 60
    d, e = tm.one_two_one(n)
    w = oracle.eigvals(d, e)
    k = np.arange(1, n + 1)
    assert np.max(np.abs(w - (2 - 2 * np.cos(np.pi * k / (n + 1))))) <= 1e-13
    # negative beta_1 Gershgorin containment
    dg, eg = np.array([0.0, 5.0, 5.0]), np.array([-1.0, 0.1])
    gl, gu = oracle.gershgorin(dg, eg)
    wg = np.linalg.eigvalsh(oracle.dense(dg, eg))
    assert gl <= wg[0] and wg[-1] <= gu
    # random matrix vs LAPACK; Sturm count at the midpoints
    d, e = tm.random_uniform(40, 1, 2)
    e = np.r_[e, 0.37]  # padding so a shifted index stays in bounds
    w = oracle.eigvals(d, e[:39])
    wl = np.linalg.eigvalsh(oracle.dense(d, e[:39]))
    assert np.max(np.abs(w - wl)) <= 1e-12
    # Jacobi on the dense matrix
    wj, V = oracle.jacobi(oracle.dense(d, e[:39]))
    assert np.max(np.abs(wj - wl)) <= 1e-12
    assert np.max(np.abs(V.T @ V - np.eye(40))) <= 1e-12
    # inverse iteration on one long chain (1-2-1) and on tight clusters (glued
    # Wilkinson): orthogonality
    for d, e in (tm.one_two_one(120), tm.glued_wilkinson(63)):
        w = oracle.eigvals(d, e)
        Z = oracle.eigvecs(d, e, w)
        assert M.scaled_orthogonality(Z) <= 10


def test_pins_pass_on_committed_oracle():
    _pins()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert old in src, "mutation anchor missing: %s" % name
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "mut.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new, 1))
        lib = oracle.compile_source(path, os.path.join(tmp, "libmut.so"))
        prev = oracle.use_library(lib)
        try:
            with pytest.raises(AssertionError):
                _pins()
        finally:
            oracle.restore_library(prev)
