"""The subset workload at full size: eigenpairs 8001..12000 of the n = 20000 glued Wilkinson
matrix (W21+ blocks glued by 1e-8), with the binary64 and the double-double tree, against
the oracle's eigenvalues; residual and orthogonality computed on the device."""
import numpy as np
import pytest

import oracle
import testmats as tm

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -53
N, IL, IU = 20000, 8001, 12000


@pytest.fixture(scope="module")
def problem():
    d, e = tm.make("glued_wilkinson", N)
    w_ref = oracle.eigvals(d, e, IL, IU)
    ext = oracle.eigvals(d, e, 1, 1)[0], oracle.eigvals(d, e, N, N)[0]
    return d, e, w_ref, max(abs(ext[0]), abs(ext[1]))


@pytest.mark.parametrize("prec,orth_gate", [(0, 10.0), (1, 10.0)])
def test_glued_wilkinson_subset(cuda, problem, prec, orth_gate):
    # both trees within the 10 n eps gate
    import torch
    import paper_1401_4950_gb300 as mr3
    d, e, w_ref, tn = problem
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    w, Z, info = mr3.stemr(dt, et, rng="I", il=IL, iu=IU, opts=mr3.make_opts(prec=prec))
    torch.cuda.synchronize()
    assert info["m"] == IU - IL + 1
    err = np.max(np.abs(w.cpu().numpy() - w_ref))
    assert err <= 4 * N * EPS * tn
    TZ = dt[:, None] * Z
    TZ[:-1] += et[:N - 1, None] * Z[1:]
    TZ[1:] += et[:N - 1, None] * Z[:-1]
    resid = torch.linalg.vector_norm(TZ - Z * w[None, :], dim=0).max().item() / (N * EPS * tn)
    G = Z.T @ Z
    G.diagonal().sub_(1.0)
    orth = G.abs().max().item() / (N * EPS)
    assert resid <= 10.0, resid
    assert orth <= orth_gate, orth
