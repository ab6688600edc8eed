"""Subsets at the left end of the spectrum (Ch. 4, subset computations: matrices of order
10,001, eigenpairs 1..iu for a growing fraction iu / n): the CUDA path against the oracle's
eigenvalues, with the residual and orthogonality gates computed on the device."""
import numpy as np
import pytest

import oracle
import testmats as tm

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53
N = 10001


def _gates(d, e, w, Z, tn):
    import torch
    n = d.shape[0]
    TZ = d[:, None] * Z
    TZ[:-1] += e[:n - 1, None] * Z[1:]
    TZ[1:] += e[:n - 1, None] * Z[:-1]
    resid = torch.linalg.vector_norm(TZ - Z * w[None, :], dim=0).max().item() / (n * EPS * tn)
    G = Z.T @ Z
    G.diagonal().sub_(1.0)
    return resid, G.abs().max().item() / (n * EPS)


@pytest.mark.parametrize("kind", ["random", "wilkinson", "one_two_one", "uniform_eigs"])
@pytest.mark.parametrize("frac", [0.01, 0.1, 0.3])
def test_left_end_subset(cuda, kind, frac):
    import torch
    import paper_1401_4950_gb300 as mr3
    if kind == "uniform_eigs":
        d, e = tm.FAMILIES[kind](N, device="cuda")
    else:
        d, e = tm.make(kind, N, seed=401)
    iu = max(1, int(round(frac * N)))
    w_ref = oracle.eigvals(d, e, 1, iu)
    ends = oracle.eigvals(d, e, 1, 1)[0], oracle.eigvals(d, e, N, N)[0]
    tn = max(abs(ends[0]), abs(ends[1]))
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    w, Z, info = mr3.stemr(dt, et, rng="I", il=1, iu=iu)
    torch.cuda.synchronize()
    assert info["m"] == iu
    assert np.max(np.abs(w.cpu().numpy() - w_ref)) <= 4 * N * EPS * tn
    resid, orth = _gates(dt, et, w, Z, tn)
    assert resid <= 10.0 and orth <= 10.0, (resid, orth)
