"""Pins of the accuracy metrics (oracle/metrics.py) that gate every GPU parity test.

Each pin is a hand-built case whose residual or orthogonality defect is known in closed
form, independently of the code under test:
  * T = tridiag(-1, 2, -1) of order 3 with its exact eigenpairs (lambda = 2 - sqrt(2), 2,
    2 + sqrt(2); textbook closed form of the 1-2-1 matrix, App. D);
  * a single eigenvector moved by t e_k: the residual is t ||(T - lambda I) e_k||, which
    involves the diagonal and exactly one of the two off-diagonal terms of T at the two
    ends, so a dropped term changes it;
  * an eigenvalue moved by delta: the residual of that column is delta exactly;
  * two columns at an angle pi/2 - theta: (Z^T Z - I) has the single off-diagonal entry
    sin(theta); a column scaled by (1 + delta): the diagonal entry 2 delta + delta^2.
The planted-mistake tests run the pins on copies of the metrics module with one plausible
mistake each and check that the pins reject it.
"""
import importlib.util
import os
import sys
import tempfile

import numpy as np
import pytest

from oracle import metrics as M

EPS = 2.0 ** -53
SRC = M.__file__
S2 = np.sqrt(2.0)
LAM = np.array([2.0 - S2, 2.0, 2.0 + S2])
ZX = np.array([[0.5, S2 / 2, 0.5],
               [S2 / 2, 0.0, -S2 / 2],
               [0.5, -S2 / 2, 0.5]])  # columns: eigenvectors of tridiag(-1, 2, -1), n = 3
D3 = np.full(3, 2.0)
E3 = np.full(2, -1.0)
TN = 2.0 + S2  # spectral norm


def _close(a, b, rtol=1e-9):
    assert abs(a - b) <= rtol * abs(b), (a, b)


def _pins(m):
    # the closed-form eigenpairs have a residual and a defect at rounding level
    assert m.scaled_residual(D3, E3, LAM, ZX, TN) <= 2.0
    assert m.scaled_orthogonality(ZX) <= 2.0
    t = 1e-9
    # column 0 moved by t e_0: (T - lambda_0 I) e_0 = (sqrt 2, -1, 0), norm t sqrt 3
    Z = ZX.copy()
    Z[0, 0] += t
    _close(m.scaled_residual(D3, E3, LAM, Z, TN), t * np.sqrt(3.0) / (3 * EPS * TN), 1e-6)
    # column 1 moved by t e_2: (T - 2 I) e_2 = (0, -1, 0), norm t (upper off-diagonal term)
    Z = ZX.copy()
    Z[2, 1] += t
    _close(m.scaled_residual(D3, E3, LAM, Z, TN), t / (3 * EPS * TN), 1e-6)
    # column 2 moved by t e_1: (T - lambda_2 I) e_1 = (-1, -sqrt 2, -1), norm 2 t
    Z = ZX.copy()
    Z[1, 2] += t
    _close(m.scaled_residual(D3, E3, LAM, Z, TN), 2 * t / (3 * EPS * TN), 1e-6)
    # eigenvalue 1 moved by delta: residual of column 1 is delta ||z_1|| = delta
    dl = 3e-10
    w = LAM.copy()
    w[1] += dl
    _close(m.scaled_residual(D3, E3, w, ZX, TN), dl / (3 * EPS * TN), 1e-6)
    # the thesis' 1-norm measures: r = t (sqrt 2, -1, 0) has 1-norm t (1 + sqrt 2);
    # ||T||_1 = 4; O is the largest off-diagonal |z_i^T z_j|
    Z = ZX.copy()
    Z[0, 0] += t
    R, O = m.thesis_R_O(D3, E3, LAM, Z)
    _close(R, t * (1.0 + S2) / 4.0, 1e-6)
    _close(O, t * S2 / 2, 1e-6)  # z_0^T z_j becomes t z_j(0); the largest |z_j(0)| is 1/sqrt 2
    # orthogonality: columns 0 and 1 of I_3 at the angle pi/2 - theta
    th = 1e-11
    Z = np.eye(3)
    Z[:, 1] = [np.sin(th), np.cos(th), 0.0]
    _close(m.scaled_orthogonality(Z), np.sin(th) / (3 * EPS), 1e-6)
    # a column of norm 1 + delta
    de = 4e-12
    Z = np.eye(3)
    Z[:, 2] *= 1.0 + de
    _close(m.scaled_orthogonality(Z), (2 * de + de * de) / (3 * EPS), 1e-4)
    # a rectangular Z (n = 5 rows, 2 columns): scaled by the number of rows
    Z = np.zeros((5, 2))
    Z[0, 0] = 1.0
    Z[:, 1] = [np.sin(th), np.cos(th), 0.0, 0.0, 0.0]
    _close(m.scaled_orthogonality(Z), np.sin(th) / (5 * EPS), 1e-6)
    # sign alignment flips exactly the columns with a negative dot product
    Zs = ZX * np.array([1.0, -1.0, 1.0])[None, :]
    assert np.array_equal(m.align_signs(ZX, Zs), ZX)


def test_metric_pins_pass():
    _pins(M)


MUTATIONS = {
    "tmul_drops_upper_offdiagonal": ("out[:-1] += e[:, None] * Z[1:]", "pass"),
    "tmul_drops_lower_offdiagonal": ("out[1:] += e[:, None] * Z[:-1]", "pass"),
    "tmul_wrong_sign": ("out[1:] += e[:, None] * Z[:-1]", "out[1:] -= e[:, None] * Z[:-1]"),
    "residual_one_norm": ("return np.linalg.norm(R, axis=0), np.abs(R).sum(axis=0)",
                          "return np.abs(R).sum(axis=0), np.abs(R).sum(axis=0)"),
    "residual_extra_n": ("r2.max(initial=0.0) / (n * EPS * tnorm)",
                         "r2.max(initial=0.0) / (n * n * EPS * tnorm)"),
    "residual_wrong_shift_sign": ("- Z * np.asarray(w)[None, :]", "+ Z * np.asarray(w)[None, :]"),
    "orth_extra_factor": ("np.abs(G).max(initial=0.0) / (n * EPS))",
                          "np.abs(G).max(initial=0.0) / (2 * n * EPS))"),
    "orth_scaled_by_columns": ("n = Z.shape[0]\n    G = Z.T @ Z", "n = Z.shape[1]\n    G = Z.T @ Z"),
    "thesis_norm_drops_term": ("t1[1:] += np.abs(e)", "pass"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_metric_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert old in src, "mutation anchor missing: %s" % name
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "metrics_mut.py")
        with open(path, "w") as f:
            f.write(src.replace(old, new, 1))
        spec = importlib.util.spec_from_file_location("metrics_mut", path)
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        sys.modules.pop("metrics_mut", None)
        with pytest.raises(AssertionError):
            _pins(mod)
