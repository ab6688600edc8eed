"""The C-ABI library builds for sm_103a, loads, exports every function declared in
include/mr3.h, and rejects invalid arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

import paper_1401_4950_gb300 as mr3

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mr3.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mr3_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("mr3_stemr", "mr3_stemr_batched", "mr3_backward", "mr3_stemr_host",
                     "mr3_stemr_batched_host"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = mr3.lib()
    for name in _declared():
        assert hasattr(L, name), name


def test_version_and_strerror():
    assert "sm_103a" in mr3.version()
    L = mr3.lib()
    assert L.mr3_strerror(0) == b"success"
    assert b"invalid" in L.mr3_strerror(-3)


def _call_stemr(n, d=1, e=1, rng=0, vl=0.0, vu=1.0, il=1, iu=1, m=True, w=1, Z=1, ldz=None):
    L = mr3.lib()
    mm = ctypes.c_int(0)
    return L.mr3_stemr(n, ctypes.c_void_p(d), ctypes.c_void_p(e), rng, vl, vu, il, iu,
                       ctypes.byref(mm) if m else None, ctypes.c_void_p(w), ctypes.c_void_p(Z),
                       ldz if ldz is not None else max(n, 1), None, None, None)


@pytest.mark.parametrize("kwargs,code", [
    (dict(n=-1), -1),
    (dict(n=4, d=0), -2),
    (dict(n=4, e=0), -3),
    (dict(n=4, rng=7), -4),
    (dict(n=4, rng=1, vl=2.0, vu=1.0), -6),
    (dict(n=4, rng=2, il=0, iu=2), -7),
    (dict(n=4, rng=2, il=3, iu=2), -8),
    (dict(n=4, rng=2, il=1, iu=5), -8),
    (dict(n=4, m=False), -9),
    (dict(n=4, w=0), -10),
    (dict(n=4, Z=0), -11),
    (dict(n=4, ldz=3), -12),
])
def test_argument_checks(kwargs, code):
    # invalid arguments are rejected on the host, before any CUDA call
    assert _call_stemr(**kwargs) == code


def test_empty_problem_needs_no_gpu():
    assert _call_stemr(0, d=0, e=0, w=0, Z=0, ldz=1) == 0


def test_backward_argument_checks():
    L = mr3.lib()
    f = L.mr3_backward
    assert f(-1, 0, None, None, 1, None, None, 1, None, None, None, None) == -1
    assert f(4, 5, None, None, 4, None, None, 4, None, None, None, None) == -2
    assert f(4, 4, ctypes.c_void_p(1), ctypes.c_void_p(1), 3, None, None, 4, ctypes.c_void_p(1),
             ctypes.c_void_p(1), None, None) == -5


def test_batched_argument_checks():
    import numpy as np
    L = mr3.lib()
    off = np.array([0, 3, 2], dtype=np.int64)  # decreasing offsets
    m = np.zeros(2, dtype=np.int32)
    rc = L.mr3_stemr_batched(2, off.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(1),
                             ctypes.c_void_p(1), 0, None, None, None, None,
                             m.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(1),
                             off.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(1), None, None,
                             None)
    assert rc == -2
