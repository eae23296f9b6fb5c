"""binary32 recompute-all: the TMA-staged kernel against the thread-staged one.

Both evaluate the same per-point arithmetic on the same staged values, so a
stage, a residual and several steps must agree bit for bit, on grids where
tiles touch the periodic edges in x and y (the TMA box reads the fill value
there and the kernel patches in the periodic images), on ragged tile counts,
and across z-chunk boundaries.  FDGB300_NO_TMA=1 at creation selects the
thread-staged kernel.
"""
import os

import numpy as np
import pytest

import oracle as O
from tests.inputs import rough_state, smooth_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


def run(shape, Q0, steps, tma):
    nz, ny, nx = shape
    old = os.environ.pop("FDGB300_NO_TMA", None)
    if not tma:
        os.environ["FDGB300_NO_TMA"] = "1"
    try:
        with fd.Solver((nx, ny, nz), dt=1e-3, algorithm="recompute_all", dtype="f32") as s:
            s.set_state(Q0)
            R = s.residual()
            s.step(steps)
            return R, s.state()
    finally:
        os.environ.pop("FDGB300_NO_TMA", None)
        if old is not None:
            os.environ["FDGB300_NO_TMA"] = old


# (nz, ny, nx): every nx a multiple of 4 (the TMA row stride rule)
@pytest.mark.parametrize("shape", [(32, 32, 32), (18, 24, 20), (70, 16, 64), (9, 6, 8), (5, 37, 36)])
@pytest.mark.parametrize("kind", ["smooth", "rough"])
def test_tma_staging_equals_thread_staging(shape, kind):
    Q0 = smooth_state(shape, seed=41) if kind == "smooth" else rough_state(shape, seed=42)
    Ra, Qa = run(shape, Q0, 3, True)
    Rb, Qb = run(shape, Q0, 3, False)
    assert np.array_equal(Ra, Rb)
    assert np.array_equal(Qa, Qb)


def test_tma_residual_close_to_oracle():
    shape = (20, 24, 28)
    Q0 = smooth_state(shape, seed=43)
    ref = O.residual(Q0)
    R, _ = run(shape, Q0, 0, True)
    for v in range(5):
        assert np.abs(R[v] - ref[v]).max() <= 2e-5 * np.abs(ref[v]).max(), v


BATCH = [
    dict(n=16, Re=1600.0, Mach=0.1, algorithm="recompute_all", tile_points=0, dt=1e-3),
    dict(n=(20, 24, 70), Re=800.0, Mach=0.25, algorithm="recompute_all", tile_points=0, dt=1e-3),
    dict(n=24, Re=400.0, Mach=0.15, algorithm="store_some", tile_points=0, dt=1.5e-3),
    dict(n=(36, 9, 10), Re=1000.0, Mach=0.3, algorithm="recompute_all", tile_points=0, dt=1e-3),
    # enough (tile, z-chunk) items that the one-block-per-SM grid gives blocks several items
    dict(n=(128, 128, 256), Re=1600.0, Mach=0.1, algorithm="recompute_all", tile_points=0, dt=1e-3),
    dict(n=(96, 96, 128), Re=2000.0, Mach=0.2, algorithm="recompute_all", tile_points=0, dt=1e-3),
    dict(n=(64, 64, 512), Re=1200.0, Mach=0.1, algorithm="recompute_all", tile_points=0, dt=1e-3),
]


def batch_states(tma, steps):
    old = os.environ.pop("FDGB300_NO_TMA", None)
    if not tma:
        os.environ["FDGB300_NO_TMA"] = "1"
    try:
        with fd.Batch(BATCH, dtype="f32") as b:
            b.step(steps)
            return [b.state(i) for i in range(len(BATCH))], b.diagnostics()
    finally:
        os.environ.pop("FDGB300_NO_TMA", None)
        if old is not None:
            os.environ["FDGB300_NO_TMA"] = old


def test_batched_tma_staging_equals_thread_staging():
    """The persistent batched kernel walks (tile, z-chunk) items of several
    instances with one ring; the ring's mbarrier phases carry over between
    items, so several items per block and instances of different sizes are
    the cases to cover."""
    a, (ka, ea) = batch_states(True, 4)
    b, (kb, eb) = batch_states(False, 4)
    for i in range(len(BATCH)):
        assert np.array_equal(a[i], b[i]), i
    assert np.array_equal(ka, kb) and np.array_equal(ea, eb)
