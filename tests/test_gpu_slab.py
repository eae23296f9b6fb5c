"""z-slab decomposition on one GPU: slabs of a grid, each a library handle with 6 ghost
planes on either side, their ghosts refreshed between steps by the exchange of
paper_1610_09146_gb300.slab (here by device copies, as all slabs live in one process;
between GPUs the same plan runs over NCCL).  The slabs' own planes together must equal
the whole-grid run bit for bit (same arithmetic at every point) and the FP64 oracle to
relative L-inf 1e-12.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402
from paper_1610_09146_gb300 import native, slab  # noqa: E402

GAMMA, MACH = 1.4, 0.1
CASES = [("store_some", "f64"), ("recompute_all", "f64"), ("store_all", "f64"), ("recompute_some", "f64"),
         ("store_none", "f64"), ("store_some", "f64dw")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


def run_slabs(nx, ny, nz, world, steps, alg, dtype, dt):
    ghost = native.fd_slab_ghost_planes(fd.ALGORITHMS[alg])
    plan = slab.check_plan(nz, world, ghost)
    slabs = [slab.DeviceSlab(nx, ny, nz, z0, m, Re=1600.0, Mach=MACH, dt=dt, algorithm=alg, dtype=dtype)
             for z0, m in plan]
    try:
        for _ in range(steps):
            slab.exchange_local(slabs)
            for s in slabs:
                s.step(1)
        return np.concatenate([s.own_state() for s in slabs], axis=1)
    finally:
        for s in slabs:
            s.close()


@pytest.mark.parametrize("alg,dtype", CASES)
def test_slabs_equal_the_whole_grid_and_the_oracle(alg, dtype):
    nx, ny, nz, world, steps, dt = 20, 18, 32, 4, 3, 1e-3
    got = run_slabs(nx, ny, nz, world, steps, alg, dtype, dt)
    with fd.Solver((nx, ny, nz), dt=dt, algorithm=alg, dtype=dtype) as s:
        s.step(steps)
        whole = s.state()
    assert np.array_equal(got, whole)
    ref = O.run(O.tgv_ic(nx, ny, nz, GAMMA, MACH), steps, dt=dt)
    assert max(np.abs(got[v] - ref[v]).max() / np.abs(ref[v]).max() for v in range(5)) <= 1e-12


def test_uneven_slabs_and_a_single_slab():
    nx, ny, nz, dt = 16, 16, 27, 1e-3
    with fd.Solver((nx, ny, nz), dt=dt, algorithm="store_some") as s:
        s.step(2)
        whole = s.state()
    assert np.array_equal(run_slabs(nx, ny, nz, 3, 2, "store_some", "f64", dt), whole)  # 9 planes each
    assert np.array_equal(run_slabs(nx, ny, nz, 4, 2, "store_some", "f64", dt), whole)  # 7, 7, 7, 6
    assert np.array_equal(run_slabs(nx, ny, nz, 1, 2, "store_some", "f64", dt), whole)  # ghosts from itself


def test_plane_copies_round_trip_and_bad_arguments():
    with fd.Solver((8, 6, 10), dt=1e-3, algorithm="store_some") as s:
        Q = s.state()
        buf = torch.empty((5, 3, 6, 8), dtype=torch.float64, device="cuda")
        native.fd_get_planes_async(s.h, 4, 3, buf.data_ptr(), 1)
        torch.cuda.synchronize()
        assert np.array_equal(buf.cpu().numpy(), Q[:, 4:7])
        native.fd_set_planes_async(s.h, 0, 3, buf.data_ptr(), 1)
        Q2 = s.state()
        assert np.array_equal(Q2[:, 0:3], Q[:, 4:7]) and np.array_equal(Q2[:, 3:], Q[:, 3:])
        with pytest.raises(fd.FdError) as e:
            native.fd_get_planes_async(s.h, 8, 3, buf.data_ptr(), 1)
        assert e.value.code == fd.FD_EINVAL
    with fd.Solver((8, 8, 8), dt=1e-3, algorithm="store_some", dtype="f32") as s:
        with pytest.raises(fd.FdError):
            native.fd_get_planes_async(s.h, 0, 1, buf.data_ptr(), 1)
    for kw in [dict(ghost=5), dict(dtype=fd.FD_F32_ACCDW), dict(z_first=32), dict(nz_local=0)]:
        args = dict(nx=8, ny=8, nz_global=32, z_first=0, nz_local=8, ghost=6, dtype=fd.FD_F64) | kw
        with pytest.raises(fd.FdError) as e:
            native.fd_slab_create(args["nx"], args["ny"], args["nz_global"], args["z_first"], args["nz_local"],
                                  args["ghost"], 1600.0, 0.1, 0.71, 1.4, 1e-3, fd.FD_STORE_SOME, args["dtype"])
        assert e.value.code == fd.FD_EINVAL
