"""Structure of the representation tree against the clustering the thesis prints
(tests/golden/clustering_rho.txt: Ch. 5 Table tab:clustering and Table
tab:clusteringdouble).  rho = largest cluster / n; rho = 1/n means no cluster at all.

The binary64 rows of criterion I were measured with LAPACK's DSTEMR; the classification criterion is
the same (reldist >= 1e-3 on classification-accuracy intervals; the automatic gaptol of
this solver is 1e-3 at these orders), and this solver's rho agrees to half a unit of the
printed second decimal.  The rows of criterion II (tree "fp64abs": gaptol 1e-3 with the
root's classification amended by absolute gaps) run with opts.abs_split on.  The mixed-precision rows are
structural (no cluster, or only the Wilkinson pairs) and are matched exactly."""
import os

import numpy as np
import pytest

import testmats as tm

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows():
    out = []
    for line in open(os.path.join(HERE, "golden", "clustering_rho.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        fam, n, tree, rho = line.split()
        out.append((fam, int(n), tree, float(rho)))
    return out


_CACHE = {}


def _matrix(fam, n):
    if fam == "wilkinson":
        return tm.make(fam, n + 1)  # the thesis' Wilkinson matrices have odd order n + 1
    if fam in ("uniform_eigs", "geometric_eigs"):
        # App. D prescribed spectra: Lanczos on diag(lambda), run on the device at these sizes
        if (fam, n) not in _CACHE:
            _CACHE[(fam, n)] = tm.FAMILIES[fam](n, device="cuda")
        return _CACHE[(fam, n)]
    return tm.make(fam, n)


@pytest.mark.parametrize("fam,n,tree,rho", _rows())
def test_clustering_matches_thesis(cuda, fam, n, tree, rho):
    import torch
    import paper_1401_4950_gb300 as mr3
    d, e = _matrix(fam, n)
    dt, et = torch.tensor(d, device="cuda"), torch.tensor(e, device="cuda")
    prec = mr3.DD if tree == "mixed" else mr3.FP64
    # criterion I: relative gaps only (the default); criterion II: the absolute-gap amendment
    opts = mr3.make_opts(prec=prec, abs_split=1 if tree == "fp64abs" else 0)
    _, _, info = mr3.stemr(dt, et, opts=opts)
    torch.cuda.synchronize()
    nn = len(d)
    ours = max(info["largest_cluster"], 1) / nn
    if tree in ("fp64", "fp64abs"):
        assert abs(ours - rho) <= 0.005, (ours, rho)
    else:
        assert round(ours * n) == round(rho * n), (ours, rho)
