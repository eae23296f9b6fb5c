"""ctypes binding of the C ABI in ``include/fdgb300.h`` (argument marshalling only).

Every function keeps the C name and argument order; pointers are passed as
integers (device addresses, e.g. ``tensor.data_ptr()``) or numpy arrays (host).
Loading fails loudly when ``libfdgb300.so`` has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

FD_OK = 0
FD_EINVAL = -1
FD_ENOMEM = -2
FD_ECUDA = -3
FD_EUNSTABLE = -4
FD_EBUSY = -5

FD_STORE_ALL = 0
FD_STORE_SOME = 1
FD_RECOMPUTE_ALL = 2
FD_RECOMPUTE_SOME = 3
FD_STORE_NONE = 4
FD_RECOMPUTE_ALL_INLINE = 5

FD_F64 = 0
FD_F32_ACCDW = 1
FD_DF64 = 2
FD_F64_DW = 3

FD_KERNEL_PRIMS = 0
FD_KERNEL_GRAD = 1
FD_KERNEL_FUSED = 2
FD_KERNEL_PRODUCTS = 3
FD_KERNEL_DERIV1 = 4
FD_KERNEL_DERIV2 = 5
FD_KERNEL_CLASSES = 6

FD_NOALLOC_MAX_POINTS = 262144
KERNEL_CLASS_NAMES = ["prims", "grad", "fused", "products", "deriv1", "deriv2"]

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class FdAlloc(ctypes.Structure):
    """``fd_alloc``: device allocator callbacks."""

    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class FdInstanceDesc(ctypes.Structure):
    """``fd_instance_desc``: one instance of a batch."""

    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Re", ctypes.c_double), ("Mach", ctypes.c_double), ("Pr", ctypes.c_double),
                ("gamma", ctypes.c_double), ("dt", ctypes.c_double),
                ("algorithm", ctypes.c_int), ("tile_points", ctypes.c_int)]


class FdRequest(ctypes.Structure):
    """``fd_request``: one solve submitted to a server."""

    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Re", ctypes.c_double), ("Mach", ctypes.c_double), ("Pr", ctypes.c_double),
                ("gamma", ctypes.c_double), ("dt", ctypes.c_double), ("steps", ctypes.c_int),
                ("dtype", ctypes.c_int), ("algorithm", ctypes.c_int), ("tile_points", ctypes.c_int),
                ("tag", ctypes.c_longlong)]


class FdResult(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_longlong), ("status", ctypes.c_int), ("steps_done", ctypes.c_int),
                ("ke", ctypes.c_double), ("enstrophy", ctypes.c_double)]


class FdServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int), ("active", ctypes.c_int), ("submitted", ctypes.c_longlong),
                ("completed", ctypes.c_longlong), ("ticks", ctypes.c_longlong),
                ("arena_bytes", ctypes.c_size_t), ("arena_used", ctypes.c_size_t)]


class FdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p

# name -> (restype, argtypes)
_SIGS = {
    "fd_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_int, ctypes.POINTER(FdAlloc), _vp]),
    "fd_step": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fd_get_state": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_int]),
    "fd_set_state": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_int]),
    "fd_get_state_async": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_int]),
    "fd_set_state_async": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_int]),
    "fd_diagnostics": (ctypes.c_int, [_vp, _dp, _dp]),
    "fd_residual": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.c_int]),
    "fd_check_finite": (ctypes.c_int, [_vp]),
    "fd_device_bytes": (ctypes.c_size_t, [_vp]),
    "fd_profile": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fd_profile_read": (ctypes.c_int, [_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "fd_residual_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double, _vp]),
    "fd_selftest_wait_timeout": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
    "fd_destroy": (ctypes.c_int, [_vp]),
    "fd_last_error": (ctypes.c_char_p, [_vp]),
    "fd_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(FdInstanceDesc), ctypes.c_int,
                                       ctypes.c_int, ctypes.POINTER(FdAlloc), _vp]),
    "fd_batch_step": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fd_batch_get_state": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int]),
    "fd_batch_set_state": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int]),
    "fd_batch_diagnostics": (ctypes.c_int, [_vp, _dp, _dp]),
    "fd_batch_count": (ctypes.c_int, [_vp]),
    "fd_batch_device_bytes": (ctypes.c_size_t, [_vp]),
    "fd_batch_profile": (ctypes.c_int, [_vp, ctypes.c_int]),
    "fd_batch_profile_read": (ctypes.c_int, [_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "fd_batch_destroy": (ctypes.c_int, [_vp]),
    "fd_batch_last_error": (ctypes.c_char_p, [_vp]),
    "fd_server_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_size_t, ctypes.c_int,
                                        ctypes.POINTER(FdAlloc), _vp]),
    "fd_server_submit": (ctypes.c_int, [_vp, ctypes.POINTER(FdRequest)]),
    "fd_server_footprint": (ctypes.c_size_t, [ctypes.POINTER(FdRequest)]),
    "fd_server_cancel": (ctypes.c_int, [_vp, ctypes.c_longlong]),
    "fd_server_tick": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "fd_server_poll": (ctypes.c_int, [_vp, ctypes.POINTER(FdResult), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "fd_slab_ghost_planes": (ctypes.c_int, [ctypes.c_int]),
    "fd_slab_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(FdAlloc), _vp]),
    "fd_get_planes_async": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int]),
    "fd_set_planes_async": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int]),
    "fd_fp64_peak": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), _vp, ctypes.c_size_t]),
    "fd_server_get_state": (ctypes.c_int, [_vp, ctypes.c_longlong, _vp, ctypes.c_size_t, ctypes.c_int]),
    "fd_server_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(FdServerStats)]),
    "fd_server_destroy": (ctypes.c_int, [_vp]),
    "fd_server_last_error": (ctypes.c_char_p, [_vp]),
}


def exported_symbols():
    """Names of the entry points this binding expects the library to export."""
    return list(_SIGS)


def lib_path() -> str:
    return LIB


def load():
    """Load the native library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_1610_09146_gb300.build.build() "
                               "(the CUDA path has no fallback)")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, h=None):
    if rc != FD_OK:
        msg = load().fd_last_error(h).decode()
        raise FdError(rc, msg)
    return rc


def _hostptr(a: np.ndarray):
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError("host buffers must be C-contiguous float64 numpy arrays")
    return a.ctypes.data


# ---- thin wrappers with the C names ------------------------------------------


def fd_create(nx, ny, nz, Re, Mach, Pr, gamma, dt, algorithm, dtype, alloc=None, stream=0):
    """Returns the handle (an opaque integer).  `alloc` is an FdAlloc or None,
    `stream` a cudaStream_t as an integer (0 = default stream)."""
    h = _vp()
    ap = ctypes.byref(alloc) if alloc is not None else None
    rc = load().fd_create(ctypes.byref(h), nx, ny, nz, Re, Mach, Pr, gamma, dt, algorithm, dtype, ap,
                          _vp(stream or None))
    _check(rc, None)
    return h.value


def fd_slab_ghost_planes(algorithm):
    return load().fd_slab_ghost_planes(algorithm)


def fd_slab_create(nx, ny, nz_global, z_first, nz_local, ghost, Re, Mach, Pr, gamma, dt, algorithm, dtype,
                   alloc=None, stream=0):
    """Handle of a z-slab (fd_slab_create); returns it as an opaque integer."""
    h = _vp()
    ap = ctypes.byref(alloc) if alloc is not None else None
    rc = load().fd_slab_create(ctypes.byref(h), nx, ny, nz_global, z_first, nz_local, ghost, Re, Mach, Pr, gamma, dt,
                               algorithm, dtype, ap, _vp(stream or None))
    _check(rc, None)
    return h.value


def fd_get_planes_async(h, z, count, dst, dst_is_device=1):
    return _check(load().fd_get_planes_async(h, z, count, dst, dst_is_device), h)


def fd_set_planes_async(h, z, count, src, src_is_device=1):
    return _check(load().fd_set_planes_async(h, z, count, src, src_is_device), h)


def fd_step(h, n):
    return _check(load().fd_step(h, n), h)


def fd_get_state(h, dst, n_elems=None, dst_is_device=None):
    """dst: numpy float64 array (host) or an int device address (then give n_elems)."""
    if isinstance(dst, np.ndarray):
        return _check(load().fd_get_state(h, _hostptr(dst), dst.size, 0), h)
    return _check(load().fd_get_state(h, dst, n_elems, 1 if dst_is_device is None else dst_is_device), h)


def fd_set_state(h, src, n_elems=None, src_is_device=None):
    if isinstance(src, np.ndarray):
        return _check(load().fd_set_state(h, _hostptr(src), src.size, 0), h)
    return _check(load().fd_set_state(h, src, n_elems, 1 if src_is_device is None else src_is_device), h)


def fd_get_state_async(h, dst, n_elems, dst_is_device):
    """Stream-ordered copy of the state to the address dst (int); returns without waiting."""
    return _check(load().fd_get_state_async(h, dst, n_elems, dst_is_device), h)


def fd_set_state_async(h, src, n_elems, src_is_device):
    """Stream-ordered replacement of the state from the address src (int)."""
    return _check(load().fd_set_state_async(h, src, n_elems, src_is_device), h)


def fd_diagnostics(h):
    ke = ctypes.c_double()
    en = ctypes.c_double()
    _check(load().fd_diagnostics(h, ctypes.byref(ke), ctypes.byref(en)), h)
    return ke.value, en.value


def fd_residual(h, dst, n_elems=None, dst_is_device=None):
    if isinstance(dst, np.ndarray):
        return _check(load().fd_residual(h, _hostptr(dst), dst.size, 0), h)
    return _check(load().fd_residual(h, dst, n_elems, 1 if dst_is_device is None else dst_is_device), h)


def fd_check_finite(h):
    return load().fd_check_finite(h)


def fd_device_bytes(h):
    return load().fd_device_bytes(h)


def fd_profile(h, enable):
    return _check(load().fd_profile(h, 1 if enable else 0), h)


def fd_profile_read(h, kernel_class):
    """(total milliseconds, launches) of one kernel class since the last fd_profile."""
    ms = ctypes.c_double()
    cnt = ctypes.c_longlong()
    _check(load().fd_profile_read(h, kernel_class, ctypes.byref(ms), ctypes.byref(cnt)), h)
    return ms.value, cnt.value


def fd_residual_noalloc(Q, R, nx, ny, nz, Re, Mach, Pr, gamma, stream=0):
    """Q, R: device addresses (ints) of caller-owned float64 arrays.  Returns the status
    code as is (no message is set by this entry point)."""
    return load().fd_residual_noalloc(Q, R, nx, ny, nz, Re, Mach, Pr, gamma, _vp(stream or None))


def fd_selftest_wait_timeout():
    """Make one bounded wait inside a kernel run out (see the header); returns the
    kernel's error word (1 when the wait gave up, as designed)."""
    w = ctypes.c_int(0)
    _check(load().fd_selftest_wait_timeout(ctypes.byref(w)), None)
    return w.value


def fd_destroy(h):
    return _check(load().fd_destroy(h), None)


def fd_last_error(h=None):
    return load().fd_last_error(h).decode()


# ---- batched instances -------------------------------------------------------


def _bcheck(rc: int, b=None):
    if rc != FD_OK:
        raise FdError(rc, load().fd_batch_last_error(b).decode())
    return rc


def fd_batch_create(descs, dtype, alloc=None, stream=0):
    """descs: sequence of FdInstanceDesc (or tuples in its field order).  Returns the batch handle."""
    arr = (FdInstanceDesc * len(descs))(*[d if isinstance(d, FdInstanceDesc) else FdInstanceDesc(*d)
                                         for d in descs])
    b = _vp()
    ap = ctypes.byref(alloc) if alloc is not None else None
    _bcheck(load().fd_batch_create(ctypes.byref(b), arr, len(descs), dtype, ap, _vp(stream or None)), None)
    return b.value


def fd_batch_step(b, n):
    return _bcheck(load().fd_batch_step(b, n), b)


def fd_batch_get_state(b, i, dst, n_elems=None, dst_is_device=None):
    if isinstance(dst, np.ndarray):
        return _bcheck(load().fd_batch_get_state(b, i, _hostptr(dst), dst.size, 0), b)
    return _bcheck(load().fd_batch_get_state(b, i, dst, n_elems, 1 if dst_is_device is None else dst_is_device), b)


def fd_batch_set_state(b, i, src, n_elems=None, src_is_device=None):
    if isinstance(src, np.ndarray):
        return _bcheck(load().fd_batch_set_state(b, i, _hostptr(src), src.size, 0), b)
    return _bcheck(load().fd_batch_set_state(b, i, src, n_elems, 1 if src_is_device is None else src_is_device), b)


def fd_batch_diagnostics(b):
    n = load().fd_batch_count(b)
    ke = np.empty(n)
    en = np.empty(n)
    _bcheck(load().fd_batch_diagnostics(b, ke.ctypes.data_as(_dp), en.ctypes.data_as(_dp)), b)
    return ke, en


def fd_batch_count(b):
    return load().fd_batch_count(b)


def fd_batch_device_bytes(b):
    return load().fd_batch_device_bytes(b)


def fd_batch_profile(b, enable):
    return _bcheck(load().fd_batch_profile(b, 1 if enable else 0), b)


def fd_batch_profile_read(b, kernel_class):
    ms = ctypes.c_double()
    cnt = ctypes.c_longlong()
    _bcheck(load().fd_batch_profile_read(b, kernel_class, ctypes.byref(ms), ctypes.byref(cnt)), b)
    return ms.value, cnt.value


def fd_batch_destroy(b):
    return _bcheck(load().fd_batch_destroy(b), None)


def fd_batch_last_error(b=None):
    return load().fd_batch_last_error(b).decode()


# ---- continuous-batching server ---------------------------------------------


def _scheck(rc: int, srv=None):
    if rc != FD_OK:
        raise FdError(rc, load().fd_server_last_error(srv).decode())
    return rc


def fd_server_create(arena_bytes, max_active, alloc=None, stream=0):
    srv = _vp()
    ap = ctypes.byref(alloc) if alloc is not None else None
    _scheck(load().fd_server_create(ctypes.byref(srv), arena_bytes, max_active, ap, _vp(stream or None)), None)
    return srv.value


def fd_server_submit(srv, req: FdRequest):
    return _scheck(load().fd_server_submit(srv, ctypes.byref(req)), srv)


def fd_server_footprint(req: FdRequest):
    return load().fd_server_footprint(ctypes.byref(req))


def fd_server_cancel(srv, tag):
    return _scheck(load().fd_server_cancel(srv, tag), srv)


def fd_server_tick(srv):
    n = ctypes.c_int()
    _scheck(load().fd_server_tick(srv, ctypes.byref(n)), srv)
    return n.value


def fd_server_poll(srv, max_results=1024):
    buf = (FdResult * max_results)()
    n = ctypes.c_int()
    _scheck(load().fd_server_poll(srv, buf, max_results, ctypes.byref(n)), srv)
    return [buf[i] for i in range(n.value)]


def fd_server_get_state(srv, tag, dst, n_elems=None, dst_is_device=None):
    """Final state of a finished, unpolled solve into dst (numpy float64 array, or a device
    pointer with n_elems and dst_is_device=1)."""
    if isinstance(dst, np.ndarray):
        return _scheck(load().fd_server_get_state(srv, tag, _hostptr(dst), dst.size, 0), srv)
    return _scheck(load().fd_server_get_state(srv, tag, dst, n_elems, 1 if dst_is_device is None else
                                              int(dst_is_device)), srv)


def fd_server_get_stats(srv):
    st = FdServerStats()
    _scheck(load().fd_server_get_stats(srv, ctypes.byref(st)), srv)
    return st


def fd_server_destroy(srv):
    return _scheck(load().fd_server_destroy(srv), None)


def fd_server_last_error(srv=None):
    return load().fd_server_last_error(srv).decode()


def fd_fp64_peak():
    """Measured binary64 FMA rate of the current device in flop/s (fd_fp64_peak)."""
    import torch
    scratch = torch.empty(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
                          * 2048, dtype=torch.float64, device="cuda")
    out = ctypes.c_double()
    rc = load().fd_fp64_peak(ctypes.byref(out), scratch.data_ptr(), scratch.numel() * 8)
    if rc != FD_OK:
        raise FdError(rc, "fd_fp64_peak failed")
    return out.value
