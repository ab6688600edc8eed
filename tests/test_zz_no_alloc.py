"""mr3_stemr_static (workspace in a fixed per-device array, no device allocation in the
call) against mr3_stemr on the same inputs, through the C ABI.  Collected last, so that it
runs both alone and after every other test has used the library.

Who needs it: a caller whose device memory is claimed in full up front by its own
allocator, or who may not enter an allocator during a solve, cannot let mr3_stemr grow
its workspace pool.  The last test checks the contract itself: after the set-up call,
a solve leaves the device's free memory unchanged."""
import numpy as np
import pytest

import testmats as tm
from _checks import EPS, check_eigenpairs, tnorm_of

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    x = np.asarray(x, dtype=np.float64)
    return torch.tensor(x if len(x) else np.zeros(1), device="cuda")


def _both(d, e, **kw):
    import torch
    import paper_1401_4950_gb300 as mr3
    dt, et = _dev(d), _dev(e)
    w0, Z0, i0 = mr3.stemr(dt, et, **kw)
    runs = []
    for _ in range(2):  # two calls in a row on the same array
        w1, Z1, i1 = mr3.stemr_static(dt, et, **kw)
        torch.cuda.synchronize()
        runs.append((w1.cpu().numpy(), Z1.cpu().numpy(), i1))
    torch.cuda.synchronize()
    return (w0.cpu().numpy(), Z0.cpu().numpy(), i0), runs


def _agree(d, e, ref, got, orth_gate=10.0):
    w0, Z0, i0 = ref
    w1, Z1, i1 = got
    n = len(d)
    tn = tnorm_of(d, e)
    assert i1["m"] == i0["m"] and w1.shape == w0.shape and Z1.shape == Z0.shape
    assert i1["status"] == i0["status"]
    if w0.size == 0:
        return
    assert np.max(np.abs(w1 - w0)) <= 4 * n * EPS * tn
    # same algorithm, same seed: the columns agree to within the eigenvector error bound
    # for separated eigenvalues, and the static result passes the parity gates itself
    g = np.minimum(np.r_[np.inf, np.diff(w0)], np.r_[np.diff(w0), np.inf])
    sep = g > 1e-3 * tn
    dz = np.abs(Z1 - Z0).max(axis=0)
    assert np.all(dz[sep] <= 1e3 * n * EPS * tn / g[sep]), dz[sep].max()
    assert abs(i1["nblocks"] - i0["nblocks"]) == 0


@pytest.mark.parametrize("kind,n", [("random", 700), ("one_two_one", 1024),
                                    ("glued_wilkinson", 420), ("clement", 301)])
def test_static_matches_stemr_twice(cuda, kind, n):
    d, e = tm.make(kind, n, seed=211)
    ref, runs = _both(d, e)
    for got in runs:
        _agree(d, e, ref, got)
        check_eigenpairs(d, e, got[0], got[1], vec_compare=False)


def test_static_split_and_subsets(cuda):
    # a matrix that splits (output sorted across blocks) and the two subset ranges
    d, e = tm.make("random", 600, seed=212)
    e = np.array(e)
    e[[99, 300, 301, 450]] = 0.0
    ref, runs = _both(d, e)
    for got in runs:
        _agree(d, e, ref, got)
        check_eigenpairs(d, e, got[0], got[1], vec_compare=False)
    ref, runs = _both(d, e, rng="I", il=37, iu=411)
    for got in runs:
        _agree(d, e, ref, got)
        check_eigenpairs(d, e, got[0], got[1], il=37, iu=411, vec_compare=False)
    ref, runs = _both(d, e, rng="V", vl=-0.5, vu=1.25)
    for got in runs:
        _agree(d, e, ref, got)


def test_static_preallocated_outputs_and_size_limit(cuda):
    import torch
    import paper_1401_4950_gb300 as mr3
    n = 257
    d, e = tm.make("random", n, seed=213)
    dt, et = _dev(d), _dev(e)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    Zb = torch.empty((n, n), dtype=torch.float64, device="cuda")
    w1, Z1, _ = mr3.stemr_static(dt, et, out=(w, Zb))
    assert w1.data_ptr() == w.data_ptr() and Z1.data_ptr() == Zb.data_ptr()
    w0, Z0, _ = mr3.stemr(dt, et)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(w1 - w0)).item() <= 4 * n * EPS * tnorm_of(d, e)
    big = mr3.STATIC_MAX_N + 1
    db, eb = _dev(np.ones(big)), _dev(np.full(big - 1, 0.5))
    with pytest.raises(mr3.Mr3Error) as ex:
        mr3.stemr_static(db, eb)
    assert ex.value.code == 7


def test_static_call_allocates_no_device_memory(cuda):
    # set-up first (n = 0 loads the kernels and the array), then outputs allocated by the
    # caller; from there on a solve must leave the device's free memory unchanged (any
    # allocation, the library's pool included once trimmed, maps at least one 2 MiB page)
    import torch
    import paper_1401_4950_gb300 as mr3
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    w_, Z_, i_ = mr3.stemr_static(empty, empty)
    assert i_["m"] == 0 and w_.numel() == 0
    n = 640
    d, e = tm.make("glued_wilkinson", n, seed=214)
    dt, et = _dev(d), _dev(e)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    Zb = torch.empty((n, n), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    mr3.release_memory()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        mr3.stemr_static(dt, et, out=(w, Zb))
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    w0, Z0, _ = mr3.stemr(dt, et)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(w - w0)).item() <= 4 * n * EPS * tnorm_of(d, e)
