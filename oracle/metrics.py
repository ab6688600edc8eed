"""Accuracy metrics for computed eigenpairs -- TEST INFRASTRUCTURE ONLY.

* scaled residual   max_i ||T z_i - lambda_i z_i||_2 / (n eps ||T||)
* scaled orthogonality  max_ij |(Z^T Z - I)_ij| / (n eps)
* the thesis' R and O (Sec. 2.4, definition of residual and orthogonality):
  R = max_i ||T z_i - lambda_i z_i||_1 / ||T||_1,  O = max_{i != j} |z_i^T z_j|
with eps = 2^-53 and ||T|| = max(|lambda_1|, |lambda_n|) (the spectral norm).
"""
from __future__ import annotations

import numpy as np

EPS = np.finfo(np.float64).eps / 2.0


def tmul(d, e, Z):
    """T @ Z for tridiagonal T = (d, e) without forming T."""
    Z = np.asarray(Z)
    out = d[:, None] * Z
    if len(d) > 1:
        out[:-1] += e[:, None] * Z[1:]
        out[1:] += e[:, None] * Z[:-1]
    return out


def residuals(d, e, w, Z):
    R = tmul(np.asarray(d), np.asarray(e)[: len(d) - 1], Z) - Z * np.asarray(w)[None, :]
    return np.linalg.norm(R, axis=0), np.abs(R).sum(axis=0)


def scaled_residual(d, e, w, Z, tnorm):
    n = len(d)
    r2, _ = residuals(d, e, w, Z)
    return float(r2.max(initial=0.0) / (n * EPS * tnorm))


def scaled_orthogonality(Z):
    n = Z.shape[0]
    G = Z.T @ Z - np.eye(Z.shape[1])
    return float(np.abs(G).max(initial=0.0) / (n * EPS))


def thesis_R_O(d, e, w, Z):
    d = np.asarray(d)
    e = np.asarray(e)[: len(d) - 1]
    t1 = np.abs(d).copy()
    if len(d) > 1:
        t1[:-1] += np.abs(e)
        t1[1:] += np.abs(e)
    tn1 = t1.max()
    _, r1 = residuals(d, e, w, Z)
    G = Z.T @ Z
    np.fill_diagonal(G, 0.0)
    return float(r1.max(initial=0.0) / tn1), float(np.abs(G).max(initial=0.0))


def align_signs(Zref, Z):
    """Flip the columns of Z so that each has a non-negative dot with Zref's column."""
    s = np.sign(np.einsum("ij,ij->j", Zref, Z))
    s[s == 0] = 1.0
    return Z * s[None, :]
