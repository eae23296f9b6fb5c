"""z-slab decomposition on the host (the paper's domain decomposition, Section 4.1).

The plan and the ghost exchange of paper_1610_09146_gb300.slab, the code the GPU
slabs use, are checked with the oracle as the solver of each slab: every slab
holds its planes plus 6 ghost planes on either side of a periodic grid; after a
ghost refresh, one oracle RK3 step of each padded slab (periodic over the slab,
with the grid's spacing) is exact on the slab's own planes, because a stage's
result at a plane reads planes within 2 of it.  The reassembled own planes must
then equal the oracle's whole-grid result bit for bit (the oracle's arithmetic at
a point does not depend on where the point sits).  Two ranks exchange over gloo;
three slabs in one process exchange by copies.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_1610_09146_gb300 import slab
from tests.inputs import smooth_state

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GHOST = 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_split_covers_the_grid_evenly():
    for nz, world in [(24, 2), (25, 3), (7, 7), (64, 5)]:
        plan = slab.split(nz, world)
        assert [z for z, _ in plan] == list(np.cumsum([0] + [m for _, m in plan])[:-1])
        assert sum(m for _, m in plan) == nz
        assert max(m for _, m in plan) - min(m for _, m in plan) <= 1
    with pytest.raises(ValueError):
        slab.split(3, 4)
    with pytest.raises(ValueError):
        slab.check_plan(24, 3, GHOST + 3)
    assert slab.neighbours(0, 3) == (2, 1) and slab.neighbours(2, 3) == (1, 0)


def test_exchange_reassembles_the_periodic_field():
    rng = np.random.default_rng(7)
    Q = rng.standard_normal((5, 25, 4, 3))
    plan = slab.check_plan(25, 3, GHOST)
    slabs = [slab.HostSlab(Q, z0, m, GHOST) for z0, m in plan]
    for s in slabs:  # stale ghosts
        s.A[:, :GHOST] = 0
        s.A[:, GHOST + s.nz_local:] = 0
    slab.exchange_local(slabs)
    for (z0, m), s in zip(plan, slabs):
        idx = np.arange(z0 - GHOST, z0 + m + GHOST) % 25
        assert np.array_equal(s.A.numpy(), Q[:, idx])


def _oracle_slab_steps(Q0, plan, steps, dt, exchange, slabs):
    n = Q0.shape[-1]
    h = (2 * np.pi / n,) * 3
    for _ in range(steps):
        exchange(slabs)
        for s in slabs:
            s.A[:] = torch.from_numpy(O.run(s.A.numpy(), 1, dt=dt, h=h))
    return np.concatenate([s.own() for s in slabs], axis=1)


def test_three_slabs_step_equals_the_whole_grid():
    n, steps, dt = 24, 3, 1e-3
    Q0 = smooth_state((n, n, n), seed=17)
    plan = slab.check_plan(n, 3, GHOST)
    slabs = [slab.HostSlab(Q0, z0, m, GHOST) for z0, m in plan]
    got = _oracle_slab_steps(Q0, plan, steps, dt, slab.exchange_local, slabs)
    assert np.array_equal(got, O.run(Q0, steps, dt=dt))


def _gloo_worker(rank, port, out):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch

    import oracle as O
    from paper_1610_09146_gb300 import slab
    from tests.inputs import smooth_state
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    n, steps, dt = 20, 2, 1e-3
    Q0 = O.tgv_ic(n, n, n, 1.4, 0.1) if out["kind"] == "tgv" else smooth_state((n, n, n), seed=23)
    z0, m = slab.check_plan(n, 2, GHOST)[rank]
    s = slab.HostSlab(Q0, z0, m, GHOST)
    s.A[:, :GHOST] = 0  # ghosts start stale: only the exchange may fill them
    s.A[:, GHOST + m:] = 0
    h = (2 * np.pi / n,) * 3
    for _ in range(steps):
        slab.exchange_dist(s, rank, 2, dist)
        s.A[:] = torch.from_numpy(O.run(s.A.numpy(), 1, dt=dt, h=h))
    mine = torch.from_numpy(np.ascontiguousarray(s.own())).reshape(-1)  # both slabs hold n / 2 planes
    bufs = [torch.empty_like(mine) for _ in range(2)]
    dist.all_gather(bufs, mine)
    if rank == 0:
        parts = [b.numpy().reshape(5, -1, n, n) for b in bufs]
        out["ok"] = bool(np.array_equal(np.concatenate(parts, axis=1), O.run(Q0, steps, dt=dt)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["tgv", "smooth"])
def test_two_gloo_ranks_step_equals_the_whole_grid(kind):
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        out["kind"] = kind
        mp.spawn(_gloo_worker, args=(port, out), nprocs=2, join=True)
        assert out.get("ok") is True
