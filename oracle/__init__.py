"""FP64 CPU oracle for the Navier-Stokes residual + low-storage RK3 of
Jammy, Jacobs & Sandham (arXiv 1610.09146), Sections 2 and 3.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the CPU
baseline leg of the benchmark are the only callers.  The CUDA product path
never imports this package and shares no code with it.

This module is a ctypes wrapper over ``fd_oracle.c`` (plain C, OpenMP over
z-planes, ``-O2 -ffp-contract=off``) plus numpy conveniences.  ``build()``
compiles the library with gcc into this directory; it is rebuilt when the
source is newer than the library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fd_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


class Params(ctypes.Structure):
    """Mirror of ``or_params``: grid sizes, spacings and the flow constants of Section 3."""

    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
        ("Re", ctypes.c_double), ("Mach", ctypes.c_double), ("Pr", ctypes.c_double),
        ("gamma", ctypes.c_double), ("dt", ctypes.c_double),
    ]


RHS_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, _dp, _dp)


def build(force: bool = False) -> str:
    """Compile ``fd_oracle.c`` into ``liboracle.so`` with gcc (OpenMP, no FP contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i, d, P = ctypes.c_int, ctypes.c_double, ctypes.POINTER(Params)
        L.or_d1.argtypes = [_dp, i, i, i, i, d, _dp]
        L.or_d2.argtypes = [_dp, i, i, i, i, d, _dp]
        L.or_tgv_ic.argtypes = [i, i, i, d, d, _dp]
        L.or_primitives.argtypes = [i, i, i, d, d, _dp, _dp]
        L.or_residual.argtypes = [P, _dp, _dp]
        L.or_rk_coefficients.argtypes = [_dp, _dp]
        L.or_rk_update.argtypes = [ctypes.c_long, i, d, _dp, _dp, _dp]
        L.or_lsrk3_step.argtypes = [ctypes.c_long, d, _dp, _dp, _dp, RHS_FN, ctypes.c_void_p]
        L.or_run.argtypes = [P, _dp, i]
        L.or_run.restype = i
        L.or_diagnostics.argtypes = [i, i, i, _dp, _dp, _dp]
        L.or_num_threads.restype = i
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _shape(f: np.ndarray):
    nz, ny, nx = f.shape[-3:]
    return nx, ny, nz


def num_threads() -> int:
    return lib().or_num_threads()


def _h(f: np.ndarray, axis: int, h):
    return 2.0 * np.pi / _shape(f)[axis] if h is None else float(h)


def d1(f: np.ndarray, axis: int, h=None) -> np.ndarray:
    """First derivative of a [z][y][x] periodic field along axis (0 = x, 1 = y, 2 = z).

    The spacing defaults to 2*pi/n along that axis."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    lib().or_d1(_ptr(f), *_shape(f), axis, _h(f, axis, h), _ptr(out))
    return out


def d2(f: np.ndarray, axis: int, h=None) -> np.ndarray:
    """Pure second derivative of a [z][y][x] periodic field along axis."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    lib().or_d2(_ptr(f), *_shape(f), axis, _h(f, axis, h), _ptr(out))
    return out


def tgv_ic(nx: int, ny: int, nz: int, gamma: float = 1.4, mach: float = 0.1) -> np.ndarray:
    """Taylor-Green vortex conservative state Q[5][nz][ny][nx]."""
    Q = np.empty((5, nz, ny, nx), dtype=np.float64)
    lib().or_tgv_ic(nx, ny, nz, gamma, mach, _ptr(Q))
    return Q


def primitives(Q: np.ndarray, gamma: float = 1.4, mach: float = 0.1) -> np.ndarray:
    """u, v, w, p, T as [5][nz][ny][nx]."""
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    out = np.empty_like(Q)
    lib().or_primitives(*_shape(Q), gamma, mach, _ptr(Q), _ptr(out))
    return out


def params(shape, Re=1600.0, Mach=0.1, Pr=0.71, gamma=1.4, dt=1e-3, h=None) -> Params:
    """Parameters for a [..][nz][ny][nx] state.  ``h`` = (hx, hy, hz) defaults to
    2*pi/n per axis (the paper's periodic cube); pass the parent grid's spacing
    when the state is a periodic block cut out of a larger grid."""
    nz, ny, nx = shape[-3:]
    if h is None:
        h = (2.0 * np.pi / nx, 2.0 * np.pi / ny, 2.0 * np.pi / nz)
    return Params(nx, ny, nz, h[0], h[1], h[2], Re, Mach, Pr, gamma, dt)


def residual(Q: np.ndarray, **kw) -> np.ndarray:
    """Residual R(Q) of the mass, momentum and energy equations, [5][nz][ny][nx]."""
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    R = np.empty_like(Q)
    P = params(Q.shape, **kw)
    lib().or_residual(ctypes.byref(P), _ptr(Q), _ptr(R))
    return R


def rk_coefficients():
    a = np.zeros(3)
    b = np.zeros(3)
    lib().or_rk_coefficients(_ptr(a), _ptr(b))
    return a, b


def lsrk3_step(q: np.ndarray, dt: float, rhs) -> np.ndarray:
    """One oracle RK3 step of dq/dt = rhs(q) for a generic Python right-hand side."""
    q = np.ascontiguousarray(q, dtype=np.float64).copy()
    n = q.size
    qs = np.empty_like(q)
    r = np.empty_like(q)

    def cb(_ctx, qp, rp):
        qv = np.ctypeslib.as_array(qp, shape=(n,))
        rv = np.ctypeslib.as_array(rp, shape=(n,))
        rv[:] = rhs(qv.copy())

    fn = RHS_FN(cb)
    lib().or_lsrk3_step(n, dt, _ptr(q), _ptr(qs), _ptr(r), fn, None)
    return q


def run(Q: np.ndarray, nsteps: int, **kw) -> np.ndarray:
    """Advance Q by nsteps RK3 steps; returns the new state (input untouched)."""
    Q = np.ascontiguousarray(Q, dtype=np.float64).copy()
    P = params(Q.shape, **kw)
    rc = lib().or_run(ctypes.byref(P), _ptr(Q), nsteps)
    if rc != 0:
        raise MemoryError("oracle run could not allocate its work arrays")
    return Q


def diagnostics(Q: np.ndarray):
    """(kinetic energy, enstrophy) density-weighted volume means."""
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    ke = ctypes.c_double()
    en = ctypes.c_double()
    lib().or_diagnostics(*_shape(Q), _ptr(Q), ctypes.byref(ke), ctypes.byref(en))
    return ke.value, en.value
