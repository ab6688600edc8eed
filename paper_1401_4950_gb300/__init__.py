"""GB300-native MRRR eigensolver for symmetric tridiagonal matrices.

Python binding of ``libmr3.so`` (C ABI in ``include/mr3.h``).  This module only
marshals arguments: every step of the solve runs in the library's CUDA kernels.  PyTorch
supplies device memory and streams.  There is no CPU fallback: if the library cannot be
built or loaded, every call raises.

Entry points (same names as the C ABI):
  stemr(d, e, ...)             -> (w, Z, info)   device tensors in, device tensors out
  stemr_host(d, e, ...)        -> (w, Z, info)   numpy in, numpy out (copies inside the call)
  stemr_batched(n_off, d, e, ...) -> (m, w, Z, z_off, info)
  stemr_batched_host(n_off, d, e, ...) -> (m, w, Z, z_off, info)  host arrays in and out
  backward(w, Z, gw, gZ)       -> (dbar, ebar)
  backward_solve(d, e, w, Z, gw, gZ) -> (dbar, ebar)   any k (subsets), O(n) per eigenpair
  eigh_tridiagonal(d, e)       -> (w, Z) differentiable (torch.autograd.Function)
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build_lib

RANGE_ALL, RANGE_VALUE, RANGE_INDEX = 0, 1, 2
FP64, DD = 0, 1
FAULT_RQI_NOCONV, FAULT_SHIFT_REJECT, FAULT_NAN_SHIFT = 0x1, 0x2, 0x4
_RANGES = {"A": RANGE_ALL, "V": RANGE_VALUE, "I": RANGE_INDEX}


class Opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("gaptol", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("max_rqi", ctypes.c_int),
                ("max_shift_tries", ctypes.c_int), ("fault_mask", ctypes.c_uint),
                ("tpe", ctypes.c_int), ("max_depth", ctypes.c_int),
                ("profile", ctypes.c_int), ("rqi_team", ctypes.c_int),
                ("bisect_warps", ctypes.c_int), ("abs_split", ctypes.c_int),
                ("erep", ctypes.c_int), ("graph", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("nblocks", ctypes.c_int), ("dmax", ctypes.c_int),
                ("nclusters", ctypes.c_int), ("largest_cluster", ctypes.c_int),
                ("new_rrr", ctypes.c_int), ("untested_rrr", ctypes.c_int),
                ("rqi_iters", ctypes.c_longlong), ("rqi_iters_max", ctypes.c_int),
                ("bisect_fallbacks", ctypes.c_int), ("sturm_steps", ctypes.c_longlong),
                ("shift_steps", ctypes.c_longlong), ("twisted_steps", ctypes.c_longlong),
                ("status_counts", ctypes.c_int * 8), ("kernel_ms", ctypes.c_double * 8),
                ("kernel_launches", ctypes.c_int * 8), ("ladder_clusters", ctypes.c_int),
                ("recomputed_rrr", ctypes.c_int), ("envelope_rrr", ctypes.c_int),
                ("graph_levels", ctypes.c_int), ("graph_runs", ctypes.c_int),
                ("graph_pool_peak", ctypes.c_longlong)]

    _ARRAYS = ("status_counts", "kernel_ms", "kernel_launches")

    def as_dict(self):
        out = {k: getattr(self, k) for k, _ in self._fields_ if k not in self._ARRAYS}
        for k in self._ARRAYS:
            out[k] = list(getattr(self, k))
        return out


_lock = threading.Lock()
_lib = None


def lib():
    """The loaded libmr3 (built in-tree on first use when missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = build_lib.build()
            L = ctypes.CDLL(path)
            vp, dp, ip = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
            c_int, c_dbl = ctypes.c_int, ctypes.c_double
            L.mr3_stemr.argtypes = [c_int, dp, dp, c_int, c_dbl, c_dbl, c_int, c_int,
                                    ctypes.POINTER(c_int), dp, dp, c_int,
                                    ctypes.POINTER(Opts), ctypes.POINTER(Info), vp]
            L.mr3_stemr.restype = c_int
            L.mr3_stemr_static.argtypes = L.mr3_stemr.argtypes
            L.mr3_stemr_static.restype = c_int
            L.mr3_stemr_host.argtypes = L.mr3_stemr.argtypes
            L.mr3_stemr_host.restype = c_int
            L.mr3_stemr_batched.argtypes = [c_int, vp, dp, dp, c_int, vp, vp, vp, vp, vp, dp,
                                            vp, dp, ctypes.POINTER(Opts),
                                            ctypes.POINTER(Info), vp]
            L.mr3_stemr_batched.restype = c_int
            L.mr3_stemr_batched_host.argtypes = L.mr3_stemr_batched.argtypes
            L.mr3_stemr_batched_host.restype = c_int
            L.mr3_backward.argtypes = [c_int, c_int, dp, dp, c_int, dp, dp, c_int, dp, dp,
                                       ctypes.POINTER(Opts), vp]
            L.mr3_backward.restype = c_int
            L.mr3_backward_solve.argtypes = [c_int, c_int, dp, dp, dp, dp, c_int, dp, dp, c_int,
                                             dp, dp, ctypes.POINTER(Opts), vp]
            L.mr3_backward_solve.restype = c_int
            L.mr3_strerror.argtypes = [c_int]
            L.mr3_strerror.restype = ctypes.c_char_p
            L.mr3_version.argtypes = []
            L.mr3_version.restype = ctypes.c_char_p
            L.mr3_release_memory.argtypes = []
            L.mr3_release_memory.restype = c_int
            _lib = L
    return _lib


class Mr3Error(RuntimeError):
    def __init__(self, code, where):
        msg = lib().mr3_strerror(code).decode()
        super().__init__("%s failed with code %d: %s" % (where, code, msg))
        self.code = code


KERNEL_GROUPS = ("prologue", "root", "bisect_root", "classify", "rqi", "shift", "refine",
                 "order")


def make_opts(prec=FP64, gaptol=0.0, seed=0, max_rqi=0, max_shift_tries=0, fault_mask=0,
              tpe=0, max_depth=0, profile=0, rqi_team=0, bisect_warps=0, abs_split=0,
              erep=0, graph=0) -> Opts:
    o = Opts()
    o.prec, o.gaptol, o.seed, o.max_rqi = prec, gaptol, seed, max_rqi
    o.max_shift_tries, o.fault_mask, o.tpe, o.max_depth = max_shift_tries, fault_mask, tpe, max_depth
    o.profile, o.rqi_team, o.bisect_warps = profile, rqi_team, bisect_warps
    # abs_split: positive = absolute-gap amendment at the root on (default off)
    o.abs_split, o.erep = int(abs_split), int(bool(erep))
    # graph: 0 = level loop in one CUDA graph for solves of 2+ matrices, 1 = always, -1 = never
    o.graph = int(graph)
    return o


def _check(rc, where, allow_status=True):
    if rc < 0 or (rc > 0 and not allow_status) or rc in (5, 6, 7):
        raise Mr3Error(rc, where)
    return rc


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _range_args(rng, n, vl, vu, il, iu):
    r = _RANGES[rng] if isinstance(rng, str) else int(rng)
    if iu is None:
        iu = n
    if r == RANGE_INDEX:
        mcap = max(iu - il + 1, 0)
    else:
        mcap = n
    return r, float(vl), float(vu), int(il), int(iu), mcap


def stemr(d, e, rng="A", vl=0.0, vu=0.0, il=1, iu=None, opts=None, stream=None):
    """Eigenpairs of tridiag(e, d, e) for device tensors d (n) and e (n-1), float64.

    Returns (w, Z, info): w of shape (m,), Z of shape (n, m) (column-major storage),
    info a dict of solver statistics and the status code."""
    torch = _torch()
    n = int(d.shape[0])
    assert d.dtype == torch.float64 and d.is_cuda and d.is_contiguous()
    if n > 1:
        assert e.dtype == torch.float64 and e.is_cuda and e.is_contiguous() and e.shape[0] >= n - 1
    r, vl, vu, il, iu, mcap = _range_args(rng, n, vl, vu, il, iu)
    w = torch.empty(max(mcap, 1), dtype=torch.float64, device=d.device)
    Zb = torch.empty((max(mcap, 1), max(n, 1)), dtype=torch.float64, device=d.device)
    m = ctypes.c_int(0)
    info = Info()
    o = opts if opts is not None else make_opts()
    rc = lib().mr3_stemr(n, ctypes.c_void_p(d.data_ptr()),
                         ctypes.c_void_p(e.data_ptr() if n > 1 else 0), r, vl, vu, il, iu,
                         ctypes.byref(m), ctypes.c_void_p(w.data_ptr()),
                         ctypes.c_void_p(Zb.data_ptr()), max(n, 1), ctypes.byref(o),
                         ctypes.byref(info), _stream_ptr(stream))
    _check(rc, "mr3_stemr")
    k = m.value
    out = info.as_dict()
    out["status"] = rc
    return w[:k], Zb[:k].T, out


def stemr_static(d, e, rng="A", vl=0.0, vu=0.0, il=1, iu=None, opts=None, stream=None,
                 out=None):
    """mr3_stemr_static: as stemr, for n <= STATIC_MAX_N, with the library's workspace in
    a fixed per-device array (the call allocates no device memory).  `out` = (w, Zbuf)
    lets the caller pass preallocated outputs: w float64 of >= n entries and Zbuf
    float64 of shape (>= n, n), row j of Zbuf receiving eigenvector j."""
    torch = _torch()
    n = int(d.shape[0])
    assert d.dtype == torch.float64 and d.is_cuda and d.is_contiguous()
    if n > 1:
        assert e.dtype == torch.float64 and e.is_cuda and e.is_contiguous() and e.shape[0] >= n - 1
    r, vl, vu, il, iu, mcap = _range_args(rng, n, vl, vu, il, iu)
    if out is None:
        w = torch.empty(max(mcap, 1), dtype=torch.float64, device=d.device)
        Zb = torch.empty((max(mcap, 1), max(n, 1)), dtype=torch.float64, device=d.device)
    else:
        w, Zb = out
        assert (w.dtype == torch.float64 and w.is_cuda and w.is_contiguous()
                and w.numel() >= mcap)
        assert (Zb.dtype == torch.float64 and Zb.is_cuda and Zb.is_contiguous()
                and Zb.shape[0] >= mcap and Zb.shape[1] == max(n, 1))
        # the library's array is the current device's: every operand lives on d's device
        assert w.device == d.device and Zb.device == d.device
    if n > 1:
        assert e.device == d.device
    m = ctypes.c_int(0)
    info = Info()
    o = opts if opts is not None else make_opts()
    with torch.cuda.device(d.device):
        rc = lib().mr3_stemr_static(n, ctypes.c_void_p(d.data_ptr()),
                                    ctypes.c_void_p(e.data_ptr() if n > 1 else 0), r, vl, vu,
                                    il, iu, ctypes.byref(m), ctypes.c_void_p(w.data_ptr()),
                                    ctypes.c_void_p(Zb.data_ptr()), max(n, 1), ctypes.byref(o),
                                    ctypes.byref(info), _stream_ptr(stream))
    _check(rc, "mr3_stemr_static")
    k = m.value
    res = info.as_dict()
    res["status"] = rc
    return w[:k], Zb[:k].T, res


STATIC_MAX_N = 1024  # MR3_STATIC_MAX_N in include/mr3.h


def stemr_host(d, e, rng="A", vl=0.0, vu=0.0, il=1, iu=None, opts=None, stream=None):
    """mr3_stemr_host on numpy arrays (host in, host out); returns (w, Z, info)."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = d.shape[0]
    e = np.ascontiguousarray(e, dtype=np.float64) if n > 1 else np.zeros(1)
    r, vl, vu, il, iu, mcap = _range_args(rng, n, vl, vu, il, iu)
    w = np.empty(max(n, 1))
    Zt = np.empty((max(n, 1), max(n, 1)))  # rows are the columns of the column-major Z
    m = ctypes.c_int(0)
    info = Info()
    o = opts if opts is not None else make_opts()
    rc = lib().mr3_stemr_host(n, d.ctypes.data_as(ctypes.c_void_p), e.ctypes.data_as(ctypes.c_void_p),
                              r, vl, vu, il, iu, ctypes.byref(m), w.ctypes.data_as(ctypes.c_void_p),
                              Zt.ctypes.data_as(ctypes.c_void_p), max(n, 1), ctypes.byref(o),
                              ctypes.byref(info), _stream_ptr(stream) if stream is not None else ctypes.c_void_p(0))
    _check(rc, "mr3_stemr_host")
    k = m.value
    out = info.as_dict()
    out["status"] = rc
    return w[:k].copy(), Zt[:k].T.copy(), out


def stemr_batched(n_off, d, e, rng="A", vl=None, vu=None, il=None, iu=None, opts=None,
                  stream=None):
    """Eigenpairs of nb packed tridiagonals.

    n_off: host int64 array (nb+1); d, e: device float64 tensors of n_off[-1] entries
    (e packed with the same offsets, last slot of each matrix unused).  Returns
    (m, w, Z, z_off, info): w packed like d, Z_b at Z[z_off[b]:] as an n_b x n_b
    column-major block."""
    torch = _torch()
    n_off = np.ascontiguousarray(n_off, dtype=np.int64)
    nb = n_off.shape[0] - 1
    sizes = np.diff(n_off)
    z_off = np.zeros(nb + 1, dtype=np.int64)
    z_off[1:] = np.cumsum(sizes * sizes)
    r = _RANGES[rng] if isinstance(rng, str) else int(rng)
    w = torch.empty(max(int(n_off[-1]), 1), dtype=torch.float64, device=d.device)
    Z = torch.empty(max(int(z_off[-1]), 1), dtype=torch.float64, device=d.device)
    m = np.zeros(max(nb, 1), dtype=np.int32)
    info = Info()
    o = opts if opts is not None else make_opts()

    def ptr(a, dt):
        if a is None:
            return ctypes.c_void_p(0)
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data_as(ctypes.c_void_p)

    keep = []
    rc = lib().mr3_stemr_batched(nb, n_off.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(e.data_ptr()), r,
                                 ptr(vl, np.float64), ptr(vu, np.float64), ptr(il, np.int32),
                                 ptr(iu, np.int32), m.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.c_void_p(w.data_ptr()),
                                 z_off.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(Z.data_ptr()),
                                 ctypes.byref(o), ctypes.byref(info), _stream_ptr(stream))
    _check(rc, "mr3_stemr_batched")
    out = info.as_dict()
    out["status"] = rc
    return m[:nb], w, Z, z_off, out


def stemr_batched_host(n_off, d, e, rng="A", vl=None, vu=None, il=None, iu=None, opts=None,
                       stream=None, out=None):
    """mr3_stemr_batched_host: the packed batch on host arrays (numpy, or pinned CPU
    tensors), copied in and out inside the call.  Returns (m, w, Z, z_off, info) with w and
    Z host arrays laid out as for stemr_batched; `out` = (w, Z) reuses caller arrays
    (float64, n_off[-1] and sum(n_b^2) entries)."""
    n_off = np.ascontiguousarray(n_off, dtype=np.int64)
    nb = n_off.shape[0] - 1
    sizes = np.diff(n_off)
    z_off = np.zeros(nb + 1, dtype=np.int64)
    z_off[1:] = np.cumsum(sizes * sizes)

    def host_ptr(a):
        if hasattr(a, "data_ptr"):  # a CPU torch tensor (pinned memory is copied fastest)
            assert a.device.type == "cpu" and a.is_contiguous() and str(a.dtype) == "torch.float64"
            return ctypes.c_void_p(a.data_ptr())
        assert a.dtype == np.float64 and a.flags.c_contiguous
        return a.ctypes.data_as(ctypes.c_void_p)

    if out is None:
        w = np.empty(max(int(n_off[-1]), 1))
        Z = np.empty(max(int(z_off[-1]), 1))
    else:
        w, Z = out
    keep = []

    def ptr(a, dt):
        if a is None:
            return ctypes.c_void_p(0)
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a.ctypes.data_as(ctypes.c_void_p)

    r = _RANGES[rng] if isinstance(rng, str) else int(rng)
    m = np.zeros(max(nb, 1), dtype=np.int32)
    info = Info()
    o = opts if opts is not None else make_opts()
    rc = lib().mr3_stemr_batched_host(nb, n_off.ctypes.data_as(ctypes.c_void_p), host_ptr(d),
                                      host_ptr(e), r, ptr(vl, np.float64), ptr(vu, np.float64),
                                      ptr(il, np.int32), ptr(iu, np.int32),
                                      m.ctypes.data_as(ctypes.c_void_p), host_ptr(w),
                                      z_off.ctypes.data_as(ctypes.c_void_p), host_ptr(Z),
                                      ctypes.byref(o), ctypes.byref(info), _stream_ptr(stream))
    _check(rc, "mr3_stemr_batched_host")
    res = info.as_dict()
    res["status"] = rc
    return m[:nb], w, Z, z_off, res


def backward(w, Z, gw=None, gZ=None, opts=None, stream=None):
    """(dbar, ebar) for upstream gradients gw (k,) and gZ (n, k) of (w, Z) = eigh(T)."""
    torch = _torch()
    n, k = int(Z.shape[0]), int(Z.shape[1])
    # Z is (n, k) with column-major storage (stride (1, ldz))
    assert Z.stride(0) == 1 or k <= 1
    ldz = Z.stride(1) if k > 1 else max(n, 1)
    dd = torch.empty(max(n, 1), dtype=torch.float64, device=Z.device)
    de = torch.empty(max(n - 1, 1), dtype=torch.float64, device=Z.device)
    gzp, ldgz = 0, max(n, 1)
    if gZ is not None:
        gZc = gZ if (gZ.stride(0) == 1) else gZ.t().contiguous().t()
        gzp, ldgz = gZc.data_ptr(), (gZc.stride(1) if k > 1 else max(n, 1))
    o = opts if opts is not None else make_opts()
    rc = lib().mr3_backward(n, k, ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(Z.data_ptr()), ldz,
                            ctypes.c_void_p(gw.data_ptr() if gw is not None else 0),
                            ctypes.c_void_p(gzp), ldgz, ctypes.c_void_p(dd.data_ptr()),
                            ctypes.c_void_p(de.data_ptr()), ctypes.byref(o), _stream_ptr(stream))
    _check(rc, "mr3_backward", allow_status=False)
    return dd[:n], de[: max(n - 1, 0)]


def backward_solve(d, e, w, Z, gw=None, gZ=None, opts=None, stream=None):
    """mr3_backward_solve: (dbar, ebar) for any number of eigenpairs (w (k,), Z (n, k) with
    column-major storage) of tridiag(e, d, e), the eigenvector part one eigenpair at a time."""
    torch = _torch()
    n, k = int(Z.shape[0]), int(Z.shape[1])
    assert Z.stride(0) == 1 or k <= 1
    ldz = Z.stride(1) if k > 1 else max(n, 1)
    dd = torch.empty(max(n, 1), dtype=torch.float64, device=Z.device)
    de = torch.empty(max(n - 1, 1), dtype=torch.float64, device=Z.device)
    gzp, ldgz = 0, max(n, 1)
    if gZ is not None:
        gZc = gZ if (gZ.stride(0) == 1) else gZ.t().contiguous().t()
        gzp, ldgz = gZc.data_ptr(), (gZc.stride(1) if k > 1 else max(n, 1))
    o = opts if opts is not None else make_opts()
    rc = lib().mr3_backward_solve(n, k, ctypes.c_void_p(d.data_ptr()),
                                  ctypes.c_void_p(e.data_ptr() if n > 1 else 0),
                                  ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(Z.data_ptr()), ldz,
                                  ctypes.c_void_p(gw.data_ptr() if gw is not None else 0),
                                  ctypes.c_void_p(gzp), ldgz, ctypes.c_void_p(dd.data_ptr()),
                                  ctypes.c_void_p(de.data_ptr()), ctypes.byref(o), _stream_ptr(stream))
    _check(rc, "mr3_backward_solve", allow_status=False)
    return dd[:n], de[: max(n - 1, 0)]


def _autograd_cls():
    torch = _torch()

    class TridiagEigh(torch.autograd.Function):
        """(w, Z) = eigh(tridiag(e, d, e)) with the hand-written backward of mr3_backward."""

        @staticmethod
        def forward(ctx, d, e):
            w, Z, _ = stemr(d.detach(), e.detach())
            ctx.save_for_backward(w, Z)
            return w, Z

        @staticmethod
        def backward(ctx, gw, gZ):
            w, Z = ctx.saved_tensors
            gZc = None if gZ is None else gZ.t().contiguous().t()
            dd, de = backward(w, Z, gw.contiguous() if gw is not None else None, gZc)
            return dd, de

    return TridiagEigh


_TE = None


def eigh_tridiagonal(d, e):
    """Differentiable eigen-decomposition (all eigenpairs) of tridiag(e, d, e)."""
    global _TE
    if _TE is None:
        _TE = _autograd_cls()
    return _TE.apply(d, e)


def version() -> str:
    return lib().mr3_version().decode()


def release_memory() -> None:
    """Return the unused device memory of the library's workspace pools to the driver
    (the pools otherwise keep it for later calls)."""
    rc = lib().mr3_release_memory()
    if rc != 0:
        raise RuntimeError("mr3_release_memory: " + lib().mr3_strerror(rc).decode())
