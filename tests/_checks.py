"""Shared parity checks for the GPU tests: the CUDA path against the CPU oracle."""
import numpy as np

import oracle
from oracle import metrics as M

EPS = oracle.EPS


def tnorm_of(d, e):
    n = len(d)
    lo = oracle.eigvals(d, e, 1, 1)[0]
    hi = oracle.eigvals(d, e, n, n)[0]
    return max(abs(lo), abs(hi))


def check_eigenpairs(d, e, w, Z, il=1, iu=None, w_ref=None, tn=None, resid_gate=10.0,
                     orth_gate=10.0, vec_compare=True):
    """Eigenvalues within 4 n eps ||T|| of the oracle's; scaled residual and orthogonality
    within the gates; well-separated eigenvectors equal to the oracle's up to sign."""
    n = len(d)
    if iu is None:
        iu = n
    if tn is None:
        tn = tnorm_of(d, e)
    tn = max(tn, np.finfo(float).tiny)
    if w_ref is None:
        w_ref = oracle.eigvals(d, e, il, iu)
    assert w.shape == w_ref.shape, (w.shape, w_ref.shape)
    err = np.max(np.abs(w - w_ref)) if w.size else 0.0
    assert err <= 4 * n * EPS * tn, "eigenvalue error %.3g > %.3g" % (err, 4 * n * EPS * tn)
    if w.size == 0:
        return {}
    assert np.all(np.diff(w) >= 0), "eigenvalues not ascending"
    res = M.scaled_residual(d, e, w, Z, tn)
    orth = M.scaled_orthogonality(Z)
    stats = {"eig_err_scaled": err / (n * EPS * tn), "resid": res, "orth": orth}
    assert res <= resid_gate, stats
    assert orth <= orth_gate, stats
    # the output sign convention: an entry of largest magnitude is positive (entries that
    # tie in exact arithmetic, as in symmetric eigenvectors, differ only by rounding)
    amax = np.abs(Z).max(axis=0)
    assert np.all(Z.max(axis=0) >= amax * (1 - 1e-13))
    if vec_compare and n <= 3000:
        Zr = oracle.eigvecs(d, e, w_ref)
        full = oracle.eigvals(d, e)
        g = np.full(len(w_ref), np.inf)
        for t, j in enumerate(range(il - 1, iu)):
            if j > 0:
                g[t] = min(g[t], full[j] - full[j - 1])
            if j < n - 1:
                g[t] = min(g[t], full[j + 1] - full[j])
        sep = g > 1e-3 * tn
        if np.any(sep):
            Za = M.align_signs(Zr, Z)
            verr = np.abs(Za - Zr).max(axis=0)
            bound = np.full(len(g), np.inf)
            np.divide(1e3 * n * EPS * tn, g, out=bound, where=g > 0)
            assert np.all(verr[sep] <= bound[sep]), (verr[sep].max(), bound[sep].min())
    return stats
