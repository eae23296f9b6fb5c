"""Batched path: many uneven instances in one persistent launch per stage.

Every instance of a batch runs the single-instance per-point code, so its state
after k steps must equal, bit for bit, the same instance advanced alone with the
same family and dtype (for both dtypes), and the binary64 batch must match the
oracle to the usual 1e-12.
"""
import numpy as np
import pytest

import oracle as O
from tests.inputs import smooth_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402
from paper_1610_09146_gb300 import native  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


SPECS = [
    dict(n=16, Re=1600.0, Mach=0.1, algorithm="recompute_all", tile_points=0, dt=1e-3),
    dict(n=(20, 24, 18), Re=800.0, Mach=0.25, algorithm="store_some", tile_points=64, dt=1e-3),
    dict(n=32, Re=3200.0, Mach=0.4, algorithm="recompute_all", tile_points=256, dt=2e-3),
    dict(n=24, Re=400.0, Mach=0.15, algorithm="store_some", tile_points=0, dt=1.5e-3),
    dict(n=(8, 9, 10), Re=1000.0, Mach=0.3, algorithm="recompute_all", tile_points=32, dt=1e-3),
]


def alone(spec, dtype, steps):
    with fd.Solver(spec["n"], Re=spec["Re"], Mach=spec["Mach"], dt=spec["dt"], algorithm=spec["algorithm"],
                   dtype=dtype) as s:
        s.step(steps)
        return s.state(), s.diagnostics()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batched_instances_equal_alone_bitwise(dtype):
    steps = 5
    with fd.Batch(SPECS, dtype=dtype) as b:
        b.step(steps)
        states = [b.state(i) for i in range(len(SPECS))]
        ke, en = b.diagnostics()
    for i, spec in enumerate(SPECS):
        Q, (ke1, en1) = alone(spec, dtype, steps)
        assert np.array_equal(states[i], Q), (dtype, i)
        assert ke[i] == ke1 and en[i] == en1, (dtype, i)


def test_batched_f64_matches_oracle():
    steps = 4
    with fd.Batch(SPECS, dtype="f64") as b:
        b.step(steps)
        states = [b.state(i) for i in range(len(SPECS))]
    for i, spec in enumerate(SPECS):
        n = spec["n"]
        nx, ny, nz = (n, n, n) if isinstance(n, int) else n
        ref = O.run(O.tgv_ic(nx, ny, nz, 1.4, spec["Mach"]), steps, dt=spec["dt"], Re=spec["Re"],
                    Mach=spec["Mach"])
        for v in range(5):
            scale = max(np.abs(ref[v]).max(), 1e-300)
            assert np.abs(states[i][v] - ref[v]).max() <= 1e-12 * scale, (i, v)


def test_odd_and_even_step_counts_and_set_state():
    # graph replay alternates two parities; 1 + 2 steps must equal 3 steps
    with fd.Batch(SPECS[:3], dtype="f32") as a, fd.Batch(SPECS[:3], dtype="f32") as b:
        a.step(3)
        b.step(1)
        b.step(2)
        for i in range(3):
            assert np.array_equal(a.state(i), b.state(i))
    # set_state on one instance restarts it from the given state, others untouched
    spec = SPECS[1]
    nx, ny, nz = spec["n"]
    Q0 = smooth_state((nz, ny, nx), seed=5)
    with fd.Batch(SPECS, dtype="f64") as b:
        b.step(2)
        before = b.state(0)
        b.set_state(1, Q0)
        b.step(2)
        after0 = b.state(0)
        got = b.state(1)
    ref = O.run(Q0, 2, dt=spec["dt"], Re=spec["Re"], Mach=spec["Mach"])
    for v in range(5):
        assert np.abs(got[v] - ref[v]).max() <= 1e-12 * np.abs(ref[v]).max()
    assert not np.array_equal(before, after0)


def test_profiled_steps_equal_graph_steps():
    with fd.Batch(SPECS, dtype="f32") as a, fd.Batch(SPECS, dtype="f32") as b:
        native.fd_batch_profile(b.b, 1)
        a.step(4)
        b.step(4)
        fused_ms, fused_n = native.fd_batch_profile_read(b.b, fd.native.FD_KERNEL_FUSED)
        grad_ms, grad_n = native.fd_batch_profile_read(b.b, fd.native.FD_KERNEL_GRAD)
        native.fd_batch_profile(b.b, 0)
        for i in range(len(SPECS)):
            assert np.array_equal(a.state(i), b.state(i))
    # two families present: per stage one SS fused + one RA fused launch, one SS gradient launch
    assert fused_n == 4 * 3 * 2 and grad_n == 4 * 3
    assert fused_ms > 0


def test_bad_descriptors_are_rejected():
    with pytest.raises(fd.FdError) as e:
        fd.Batch([dict(n=16, algorithm="store_all")], dtype="f32")
    assert e.value.code == fd.FD_EINVAL
    with pytest.raises(fd.FdError):
        fd.Batch([dict(n=16, tile_points=8)], dtype="f32")
    with pytest.raises(fd.FdError):
        fd.Batch([dict(n=4)], dtype="f32")


def test_mixed_batch_equals_alone_and_the_oracle():
    """Mixed binary64 / double-word store-some batch (dtype f64dw): each instance equals
    itself run alone bit for bit, and the oracle to relative L-inf 1e-12."""
    steps = 4
    specs = [dict(s, algorithm="store_some") for s in SPECS]
    with fd.Batch(specs, dtype="f64dw") as b:
        b.step(steps)
        states = [b.state(i) for i in range(len(specs))]
        ke, en = b.diagnostics()
        Q0 = smooth_state((10, 9, 8), seed=71)
        b.set_state(4, Q0)  # set / get of a binary64 state is exact
        assert np.array_equal(b.state(4), Q0)
    for i, spec in enumerate(specs):
        Q, (ke1, en1) = alone(spec, "f64dw", steps)
        assert np.array_equal(states[i], Q), i
        assert ke[i] == ke1 and en[i] == en1, i
        n = spec["n"]
        nx, ny, nz = (n, n, n) if isinstance(n, int) else n
        ref = O.run(O.tgv_ic(nx, ny, nz, 1.4, spec["Mach"]), steps, dt=spec["dt"], Re=spec["Re"], Mach=spec["Mach"])
        assert max(np.abs(Q[v] - ref[v]).max() / np.abs(ref[v]).max() for v in range(5)) <= 1e-12, i
    with pytest.raises(fd.FdError):
        fd.Batch([dict(SPECS[0], algorithm="recompute_all")], dtype="f64dw")
