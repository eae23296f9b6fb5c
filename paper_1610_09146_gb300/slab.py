"""z-slab domain decomposition (the paper's MPI decomposition, Section 4.1).

A periodic grid of nz planes is split into `world` slabs of consecutive planes;
slab r keeps `ghost` copies of its neighbours' planes on either side, so one RK3
step of the slab is exact on its own planes without any exchange inside the step
(a stage reads planes within 2 of the point, fd_slab_ghost_planes gives 3 x 2).
Between steps every slab refreshes its ghost planes: it sends its lowest `ghost`
own planes to the slab below (they become that slab's upper ghosts) and its
highest to the slab above (that slab's lower ghosts); the neighbours wrap around
periodically.  This module holds the plan and the exchange, written once for any
slab object that can hand out and take in planes:

  own_low(g), own_high(g)        the g lowest / highest own planes, [5][g][ny][nx]
  set_ghost_low(buf), set_ghost_high(buf)   replace the g lower / upper ghost planes

HostSlab keeps a padded slab in a numpy array (host computation, tests);
DeviceSlab is a library handle (fd_slab_create) whose planes move with
fd_get_planes_async / fd_set_planes_async on its stream.  Transports:
exchange_local (every slab in this process: copies) and exchange_dist
(torch.distributed point-to-point with the two neighbours; NCCL between GPUs,
gloo between host processes).
"""
from __future__ import annotations

import numpy as np


def split(nz: int, world: int):
    """Planes of each slab: a list of (z_first, nz_local), as even as possible, in order."""
    if world < 1 or nz < world:
        raise ValueError(f"cannot split {nz} planes into {world} slabs")
    base, extra = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        m = base + (1 if r < extra else 0)
        out.append((z, m))
        z += m
    return out


def neighbours(rank: int, world: int):
    """(lower, upper) slab of `rank` on the periodic ring."""
    return (rank - 1) % world, (rank + 1) % world


def check_plan(nz: int, world: int, ghost: int):
    """The exchange sends a slab's `ghost` outermost own planes to each neighbour, so every
    slab needs at least `ghost` own planes."""
    plan = split(nz, world)
    if min(m for _, m in plan) < ghost:
        raise ValueError(f"{world} slabs of {nz} planes leave fewer than {ghost} own planes on a slab")
    return plan


def exchange_local(slabs):
    """Ghost refresh of slabs that all live in this process (list in slab order)."""
    world = len(slabs)
    lows = [s.own_low(s.ghost) for s in slabs]
    highs = [s.own_high(s.ghost) for s in slabs]
    for r, s in enumerate(slabs):
        lo, hi = neighbours(r, world)
        s.set_ghost_low(highs[lo])   # the lower neighbour's highest own planes
        s.set_ghost_high(lows[hi])   # the upper neighbour's lowest own planes


def exchange_dist(slab, rank: int, world: int, dist):
    """Ghost refresh of this process's slab with torch.distributed point-to-point messages
    to and from the two neighbours (batched, so the ring cannot deadlock).  Messages
    travel down (own lowest planes -> lower neighbour's upper ghosts) and up (own highest
    -> upper neighbour's lower ghosts); every rank posts them in the same order (down
    send, down receive, up send, up receive) and with a tag per direction, so that with
    two slabs, where both neighbours are the same rank, each message meets its receive."""
    if world == 1:
        exchange_local([slab])
        return
    import torch
    down, up = 1, 2
    lo, hi = neighbours(rank, world)
    send_low = slab.own_low(slab.ghost)
    send_high = slab.own_high(slab.ghost)
    recv_high = torch.empty_like(send_low)
    recv_low = torch.empty_like(send_high)
    ops = [dist.P2POp(dist.isend, send_low, lo, tag=down), dist.P2POp(dist.irecv, recv_high, hi, tag=down),
           dist.P2POp(dist.isend, send_high, hi, tag=up), dist.P2POp(dist.irecv, recv_low, lo, tag=up)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    slab.set_ghost_low(recv_low)
    slab.set_ghost_high(recv_high)


class HostSlab:
    """A padded slab in host memory: array [5][ghost + nz_local + ghost][ny][nx] of planes
    z_first - ghost .. z_first + nz_local + ghost - 1 (mod nz) of a periodic grid, held as
    a torch CPU tensor (so that torch.distributed can send its planes)."""

    def __init__(self, Q_global, z_first: int, nz_local: int, ghost: int):
        import torch
        nz = Q_global.shape[1]
        idx = (np.arange(z_first - ghost, z_first + nz_local + ghost)) % nz
        self.A = torch.from_numpy(np.ascontiguousarray(Q_global[:, idx]))
        self.z_first, self.nz_local, self.ghost = z_first, nz_local, ghost

    def own(self):
        g = self.ghost
        return self.A[:, g:g + self.nz_local].numpy()

    def own_low(self, g):
        return self.A[:, self.ghost:self.ghost + g].contiguous()

    def own_high(self, g):
        e = self.ghost + self.nz_local
        return self.A[:, e - g:e].contiguous()

    def set_ghost_low(self, buf):
        self.A[:, :self.ghost] = buf

    def set_ghost_high(self, buf):
        e = self.ghost + self.nz_local
        self.A[:, e:] = buf


class DeviceSlab:
    """One slab as a library handle (fd_slab_create) on the current CUDA device; its planes
    move through CUDA tensors with fd_get_planes_async / fd_set_planes_async on the
    handle's stream (the torch stream current at creation, by default)."""

    def __init__(self, nx, ny, nz_global, z_first, nz_local, ghost=None, Re=1600.0, Mach=0.1, Pr=0.71, gamma=1.4,
                 dt=None, algorithm="store_some", dtype="f64", stream=None):
        import torch

        from . import ALGORITHMS, DTYPES, dt_for_grid, native, torch_allocator
        alg = ALGORITHMS[algorithm] if isinstance(algorithm, str) else int(algorithm)
        self.ghost = native.fd_slab_ghost_planes(alg) if ghost is None else int(ghost)
        self.nx, self.ny, self.nz_local, self.z_first = nx, ny, nz_local, z_first
        self.nz = nz_local + 2 * self.ghost
        self.dt = dt_for_grid(max(nx, ny, nz_global)) if dt is None else float(dt)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.torch_stream = stream if hasattr(stream, "cuda_stream") else None
        self.stream = int(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
        self._alloc = torch_allocator()
        self.h = native.fd_slab_create(nx, ny, nz_global, z_first, nz_local, self.ghost, Re, Mach, Pr, gamma, self.dt,
                                       alg, DTYPES[dtype] if isinstance(dtype, str) else int(dtype), self._alloc,
                                       self.stream)

    def _planes(self, z, count):
        import torch

        from . import native
        buf = torch.empty((5, count, self.ny, self.nx), dtype=torch.float64, device="cuda")
        native.fd_get_planes_async(self.h, z, count, buf.data_ptr(), 1)
        return buf

    def own_low(self, g):
        return self._planes(self.ghost, g)

    def own_high(self, g):
        return self._planes(self.ghost + self.nz_local - g, g)

    def set_ghost_low(self, buf):
        from . import native
        buf = buf.contiguous()
        native.fd_set_planes_async(self.h, 0, self.ghost, buf.data_ptr(), 1)
        self._keep = getattr(self, "_keep", []) + [buf]

    def set_ghost_high(self, buf):
        from . import native
        buf = buf.contiguous()
        native.fd_set_planes_async(self.h, self.ghost + self.nz_local, self.ghost, buf.data_ptr(), 1)
        self._keep = getattr(self, "_keep", []) + [buf]

    def step(self, n: int = 1):
        """n RK3 steps; only the own planes are exact afterwards (refresh the ghosts first)."""
        from . import native
        native.fd_step(self.h, n)
        self._keep = []  # the copies that read these buffers precede the step on the stream

    def own_state(self):
        """The own planes [5][nz_local][ny][nx] as a host numpy array."""
        from . import native
        out = np.empty((5, self.nz, self.ny, self.nx))
        native.fd_get_state(self.h, out)
        return np.ascontiguousarray(out[:, self.ghost:self.ghost + self.nz_local])

    def close(self):
        from . import native
        if getattr(self, "h", None):
            native.fd_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
