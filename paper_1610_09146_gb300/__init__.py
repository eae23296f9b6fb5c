"""GB300 (sm_103a) explicit finite-difference compressible Navier-Stokes solver.

The method is that of Jammy, Jacobs & Sandham, "Performance evaluation of
explicit finite difference algorithms with varying amounts of computational
and memory intensity" (arXiv 1610.09146): fourth-order central differences,
skew-symmetric convection, viscous terms expanded to second derivatives and a
low-storage three-stage Runge-Kutta scheme on the periodic Taylor-Green
vortex (Sections 2 and 3), in the paper's store-all (BL), store-some (SS)
and recompute-all (RA) algorithm families.

All arithmetic runs in the CUDA kernels of ``libfdgb300.so`` behind the C ABI
of ``include/fdgb300.h``; this package only marshals arguments.  PyTorch
provides device memory (through the allocator callbacks) and streams.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import native
from .native import (FD_DF64, FD_EBUSY, FD_ECUDA, FD_EINVAL, FD_ENOMEM, FD_EUNSTABLE, FD_F32_ACCDW, FD_F64, FD_F64_DW,
                     FD_OK, FD_RECOMPUTE_ALL, FD_RECOMPUTE_SOME, FD_STORE_ALL, FD_STORE_NONE, FD_STORE_SOME, FdAlloc, FdError, fd_check_finite, fd_create,
                     fd_destroy, fd_device_bytes, fd_diagnostics, fd_get_state, fd_last_error, fd_residual,
                     fd_set_state, fd_step)

ALGORITHMS = {"store_all": FD_STORE_ALL, "store_some": FD_STORE_SOME, "recompute_all": FD_RECOMPUTE_ALL,
              "recompute_some": FD_RECOMPUTE_SOME, "store_none": FD_STORE_NONE,
              "recompute_all_inline": native.FD_RECOMPUTE_ALL_INLINE,
              "BL": FD_STORE_ALL, "SS": FD_STORE_SOME, "RA": FD_RECOMPUTE_ALL, "RS": FD_RECOMPUTE_SOME,
              "SN": FD_STORE_NONE, "RAI": native.FD_RECOMPUTE_ALL_INLINE}
DTYPES = {"f64": FD_F64, "f32": FD_F32_ACCDW, "f32_accdw": FD_F32_ACCDW, "df64": FD_DF64, "f64dw": FD_F64_DW}

from .workloads import dt_for_grid  # noqa: E402  (Section 3 time-step rule)

# Section 3: time step 3.385e-3 on 64^3, halved for each doubling of the grid.
DT_64 = 3.385e-3


def build(force: bool = False, verbose: bool = False) -> str:
    from .build import build as _b
    return _b(force=force, verbose=verbose)


_torch_alloc_keep = []


def torch_allocator() -> FdAlloc:
    """Allocator callbacks backed by PyTorch's CUDA caching allocator."""
    import torch

    def _alloc(ctx, nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=torch.cuda.current_device(),
                                                      stream=int(stream or 0))
        except Exception:  # an out-of-memory error becomes a NULL return (FD_ENOMEM)
            return None

    def _free(ctx, ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    a = FdAlloc(native.ALLOC_FN(_alloc), native.FREE_FN(_free), None)
    _torch_alloc_keep.append(a)  # the callbacks must outlive every handle using them
    return a


class Batch:
    """Many Taylor-Green instances advanced together (see fd_batch_* in include/fdgb300.h).

    instances: sequence of dicts with keys n (int or (nx, ny, nz)), Re, Mach, Pr, gamma, dt,
    algorithm ("store_some" | "recompute_all"), tile_points; missing keys take the defaults
    of Solver.  dtype: "f64" | "f32" for the whole batch."""

    def __init__(self, instances, dtype="f32", stream=None, use_torch_allocator=True):
        import torch
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        self.shapes = []
        descs = []
        for spec in instances:
            n = spec.get("n", 32)
            nx, ny, nz = (n, n, n) if isinstance(n, int) else tuple(n)
            alg = spec.get("algorithm", "recompute_all")
            alg = ALGORITHMS[alg] if isinstance(alg, str) else int(alg)
            dt = spec.get("dt")
            dt = dt_for_grid(max(nx, ny, nz)) if dt is None else float(dt)
            descs.append(native.FdInstanceDesc(nx, ny, nz, spec.get("Re", 1600.0), spec.get("Mach", 0.1),
                                               spec.get("Pr", 0.71), spec.get("gamma", 1.4), dt, alg,
                                               int(spec.get("tile_points", 0))))
            self.shapes.append((nz, ny, nx))
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.stream = int(stream)
        self._alloc = torch_allocator() if use_torch_allocator else None
        self.b = native.fd_batch_create(descs, self.dtype, self._alloc, self.stream)

    def __len__(self):
        return len(self.shapes)

    def step(self, n: int = 1):
        native.fd_batch_step(self.b, n)

    def state(self, i):
        out = np.empty((5,) + self.shapes[i])
        native.fd_batch_get_state(self.b, i, out)
        return out

    def set_state(self, i, src):
        native.fd_batch_set_state(self.b, i, np.ascontiguousarray(src, dtype=np.float64))

    def diagnostics(self):
        return native.fd_batch_diagnostics(self.b)

    def device_bytes(self):
        return native.fd_batch_device_bytes(self.b)

    def close(self):
        if getattr(self, "b", None):
            native.fd_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Continuous-batching server (fd_server_* in include/fdgb300.h).

    submit(dict) queues a solve (keys: n, steps, Re, Mach, Pr, gamma, dt, dtype, algorithm,
    tile_points, tag); tick() admits what fits, advances every active solve by its steps for
    the tick and retires the solves the previous tick finished (one tick stays in flight; a
    tick that leaves no solve active retires its own at once); poll() returns finished
    results as dicts."""

    def __init__(self, arena_bytes, max_active=256, stream=None, use_torch_allocator=True):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.stream = int(stream)
        self._alloc = torch_allocator() if use_torch_allocator else None
        self.s = native.fd_server_create(int(arena_bytes), int(max_active), self._alloc, self.stream)

    @staticmethod
    def request(spec) -> "native.FdRequest":
        n = spec["n"]
        nx, ny, nz = (n, n, n) if isinstance(n, int) else tuple(n)
        alg = spec.get("algorithm", "recompute_all")
        alg = ALGORITHMS[alg] if isinstance(alg, str) else int(alg)
        dt = spec.get("dt")
        dt = dt_for_grid(max(nx, ny, nz)) if dt is None else float(dt)
        dtype = spec.get("dtype", "f32")
        dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        return native.FdRequest(nx, ny, nz, spec.get("Re", 1600.0), spec.get("Mach", 0.1), spec.get("Pr", 0.71),
                                spec.get("gamma", 1.4), dt, int(spec["steps"]), dtype, alg,
                                int(spec.get("tile_points", 0)), int(spec.get("tag", 0)))

    def submit(self, spec):
        native.fd_server_submit(self.s, self.request(spec))

    def footprint(self, spec) -> int:
        return native.fd_server_footprint(self.request(spec))

    def cancel(self, tag):
        native.fd_server_cancel(self.s, tag)

    def tick(self) -> int:
        return native.fd_server_tick(self.s)

    def poll(self):
        """Finished results (the next tick releases each polled solve's memory and state)."""
        return [dict(tag=r.tag, status=r.status, steps=r.steps_done, ke=r.ke, enstrophy=r.enstrophy)
                for r in native.fd_server_poll(self.s)]

    def state(self, tag, shape):
        """Final state [5][nz][ny][nx] of a finished solve, until the first tick after its
        result was polled (shape = its grid as given in the request: n or (nx, ny, nz))."""
        nx, ny, nz = (shape, shape, shape) if isinstance(shape, int) else tuple(shape)
        out = np.empty((5, nz, ny, nx), dtype=np.float64)
        native.fd_server_get_state(self.s, int(tag), out)
        return out

    def stats(self):
        st = native.fd_server_get_stats(self.s)
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if getattr(self, "s", None):
            native.fd_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Solver:
    """One Taylor-Green instance on an nx x ny x nz periodic grid.

    algorithm: "store_all" | "store_some" | "recompute_all" | "recompute_some" | "store_none"
               (or "BL" | "SS" | "RA" | "RS" | "SN")
    dtype: "f64" | "f32" (binary32 stencils, compensated double-word state, binary64
           reductions) | "df64" (double-word arithmetic on the binary32 pipe) | "f64dw"
           (store-some only: binary64 state, pressure and RK update, double-word stencils)
    stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (current torch stream)
    """

    def __init__(self, n, Re=1600.0, Mach=0.1, Pr=0.71, gamma=1.4, dt=None, algorithm="store_some",
                 dtype="f64", stream=None, use_torch_allocator=True):
        nx, ny, nz = (n, n, n) if isinstance(n, int) else tuple(n)
        self.shape = (nz, ny, nx)
        self.dt = dt_for_grid(max(nx, ny, nz)) if dt is None else float(dt)
        self.algorithm = ALGORITHMS[algorithm] if isinstance(algorithm, str) else int(algorithm)
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.stream = int(stream)
        self._alloc = torch_allocator() if use_torch_allocator else None
        self.h = fd_create(nx, ny, nz, Re, Mach, Pr, gamma, self.dt, self.algorithm, self.dtype, self._alloc,
                           self.stream)

    @property
    def n_elems(self) -> int:
        return 5 * math.prod(self.shape)

    def step(self, n: int = 1):
        fd_step(self.h, n)

    def state(self, out=None):
        """The conserved state [5][nz][ny][nx] as a host numpy array, or into `out`
        (a numpy array, or a CUDA float64 torch tensor)."""
        if out is None:
            out = np.empty((5,) + self.shape)
        if isinstance(out, np.ndarray):
            fd_get_state(self.h, out)
        else:
            fd_get_state(self.h, out.data_ptr(), out.numel(), 1)
        return out

    def set_state(self, src):
        if isinstance(src, np.ndarray):
            fd_set_state(self.h, np.ascontiguousarray(src, dtype=np.float64))
        else:
            fd_set_state(self.h, src.data_ptr(), src.numel(), 1)

    def residual(self, out=None):
        if out is None:
            out = np.empty((5,) + self.shape)
        if isinstance(out, np.ndarray):
            fd_residual(self.h, out)
        else:
            fd_residual(self.h, out.data_ptr(), out.numel(), 1)
        return out

    def diagnostics(self):
        """(kinetic energy, enstrophy) of the current state."""
        return fd_diagnostics(self.h)

    def history(self, steps_per_sample: int, samples: int):
        """Kinetic energy and enstrophy every steps_per_sample RK3 steps (Section 3,
        Fig. 3): arrays t, ke, enstrophy of samples + 1 entries, starting with the
        current state at t = 0 (t in units of this solver's time step dt)."""
        t, ke, en = [0.0], [], []
        k, e = self.diagnostics()
        ke.append(k)
        en.append(e)
        for i in range(samples):
            self.step(steps_per_sample)
            k, e = self.diagnostics()
            t.append((i + 1) * steps_per_sample * self.dt)
            ke.append(k)
            en.append(e)
        return np.array(t), np.array(ke), np.array(en)

    def check_finite(self) -> bool:
        return fd_check_finite(self.h) == FD_OK

    def device_bytes(self) -> int:
        return fd_device_bytes(self.h)

    def close(self):
        if getattr(self, "h", None):
            fd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
