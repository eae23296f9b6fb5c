"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Tolerances (binary64 path): relative L-inf <= 1e-12 per conserved variable,
normalised by max|oracle| of that variable, after 10 steps; the residual
itself to the same bound.  Variants agree with one another to the same bound
(Section 3: all algorithms match BL "up to machine precision"; they round in
different orders, e.g. a product formed at each tap vs a stored product, and
the smallest variable, rho w, starts at zero).
Inputs are the oracle's own Taylor-Green state or seeded random fields from
tests/inputs.py; no oracle input or expected value comes from the GPU.
"""
import numpy as np
import pytest

import oracle as O
from tests.inputs import rough_state, smooth_state
from tests.sampled import oracle_one_step_at

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402

VARIANTS = ["store_all", "store_some", "recompute_all", "recompute_some", "store_none"]
GAMMA, MACH, RE, PR = 1.4, 0.1, 1600.0, 0.71


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


def rel_linf(a, b):
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(5))


def solver(shape, alg, dtype="f64", dt=1e-3, **kw):
    nz, ny, nx = shape
    return fd.Solver((nx, ny, nz), Re=kw.get("Re", RE), Mach=kw.get("Mach", MACH), Pr=PR, gamma=GAMMA, dt=dt,
                     algorithm=alg, dtype=dtype)


# ------------------------------------------------------------ initial condition


@pytest.mark.parametrize("shape", [(32, 32, 32), (20, 24, 28), (5, 5, 5)])
def test_initial_condition_matches_oracle(shape):
    nz, ny, nx = shape
    ref = O.tgv_ic(nx, ny, nz, GAMMA, MACH)
    with solver(shape, "store_some") as s:
        Q = s.state()
    assert np.abs(Q - ref).max() < 1e-13


# -------------------------------------------------------------------- residual


@pytest.mark.parametrize("alg", VARIANTS)
@pytest.mark.parametrize("shape,kind", [((23, 19, 21), "rough"), ((32, 32, 32), "smooth"), ((5, 6, 7), "rough")])
def test_residual_matches_oracle(alg, shape, kind):
    Q0 = rough_state(shape, seed=5) if kind == "rough" else smooth_state(shape, seed=6)
    ref = O.residual(Q0, Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA)
    with solver(shape, alg) as s:
        s.set_state(Q0)
        R = s.residual()
    assert rel_linf(R, ref) <= 1e-12


# --------------------------------------------------------------- 10 RK3 steps


@pytest.mark.parametrize("alg", VARIANTS)
def test_ten_steps_tgv_32_matches_oracle(alg):
    n = 32
    ref = O.run(O.tgv_ic(n, n, n, GAMMA, MACH), 10, dt=1e-3)
    with solver((n, n, n), alg) as s:
        s.step(10)
        Q = s.state()
    assert rel_linf(Q, ref) <= 1e-12


@pytest.mark.parametrize("alg", VARIANTS)
def test_ten_steps_random_ragged_grid_matches_oracle(alg):
    shape = (18, 24, 20)  # nz, ny, nx: no axis a multiple of the block size
    Q0 = smooth_state(shape, seed=21)
    ref = O.run(Q0, 10, dt=1e-3)
    with solver(shape, alg) as s:
        s.set_state(Q0)
        s.step(10)
        Q = s.state()
    assert rel_linf(Q, ref) <= 1e-12


def test_variants_agree_to_machine_precision():
    n = 32
    out = {}
    for alg in VARIANTS:
        with solver((n, n, n), alg) as s:
            s.step(10)
            out[alg] = s.state()
    for alg in VARIANTS[1:]:
        assert rel_linf(out[alg], out["store_all"]) <= 1e-12, alg


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_paper_literal_families_agree_bitwise(dtype):
    """BL, RS and SN evaluate every derivative with the same operations (work
    array, re-evaluation per equation, thread-local variable); only where the
    values live differs, so the three runs are identical bit for bit."""
    shape = (18, 24, 20)
    Q0 = smooth_state(shape, seed=33)
    out = {}
    for alg in ("store_all", "recompute_some", "store_none"):
        with solver(shape, alg, dtype=dtype) as s:
            s.set_state(Q0)
            R = s.residual()
            s.step(3)
            out[alg] = (R, s.state())
    for alg in ("recompute_some", "store_none"):
        assert np.array_equal(out[alg][0], out["store_all"][0]), alg
        assert np.array_equal(out[alg][1], out["store_all"][1]), alg


# ----------------------------------------------------------------- diagnostics


@pytest.mark.parametrize("steps", [0, 10])
def test_diagnostics_match_oracle(steps):
    n = 32
    Q = O.tgv_ic(n, n, n, GAMMA, MACH)
    Q = O.run(Q, steps, dt=1e-3) if steps else Q
    ke_ref, en_ref = O.diagnostics(Q)
    with solver((n, n, n), "store_some") as s:
        s.set_state(Q)
        ke, en = s.diagnostics()
        ke2, en2 = s.diagnostics()
    assert abs(ke - ke_ref) <= 1e-13 * ke_ref
    assert abs(en - en_ref) <= 1e-13 * en_ref
    assert (ke, en) == (ke2, en2)  # fixed reduction order: bitwise repeatable


def test_initial_kinetic_energy_closed_form_on_gpu():
    with solver((64, 64, 64), "recompute_all") as s:
        ke, en = s.diagnostics()
    h = 2 * np.pi / 64
    k1 = (8 * np.sin(h) - np.sin(2 * h)) / (6 * h)
    assert abs(ke - 0.125) < 1e-14
    assert abs(en - k1**2 * (3 / 8 - 5 * GAMMA * MACH**2 / 128)) < 1e-14


# ------------------------------------------------- full size, sampled points


@pytest.mark.slow
@pytest.mark.parametrize("alg", VARIANTS)
def test_full_size_256_one_step_sampled(alg):
    n = 256
    dt = fd.dt_for_grid(n)
    Q0 = O.tgv_ic(n, n, n, GAMMA, MACH)
    rng = np.random.default_rng(256)
    pts = [tuple(rng.integers(0, n, 3)) for _ in range(24)] + [(0, 0, 0), (n - 1, n - 1, n - 1), (1, n - 2, 0)]
    h = (2 * np.pi / n,) * 3
    ref = oracle_one_step_at(Q0, pts, dt, h)
    scale = np.abs(Q0).reshape(5, -1).max(axis=1)
    scale[3] = np.abs(ref[:, 3]).max()
    with solver((n, n, n), alg, dt=dt) as s:
        Qi = s.state()
        assert np.abs(Qi - Q0).max() < 1e-13  # initial condition, every point
        s.step(1)
        Q = s.state()
        # conservation of mass and momentum at full size
        for v in range(3):
            assert abs(Q[v].sum() - Q0[v].sum()) <= 1e-12 * np.abs(Q0[v]).sum() + 1e-9
    got = np.array([Q[:, z, y, x] for (z, y, x) in pts])
    for v in range(5):
        assert np.abs(got[:, v] - ref[:, v]).max() <= 1e-12 * scale[v], v


# ------------------------------------------------------------------ edge cases


@pytest.mark.parametrize("alg", VARIANTS)
def test_smallest_grid_and_zero_steps(alg):
    shape = (5, 5, 5)
    Q0 = smooth_state(shape, seed=2)
    ref = O.run(Q0, 3, dt=1e-3)
    with solver(shape, alg) as s:
        s.set_state(Q0)
        s.step(0)
        assert np.array_equal(s.state(), Q0)
        s.step(3)
        assert rel_linf(s.state(), ref) <= 1e-12


def test_checkpoint_resume_is_bitwise():
    n = 24
    with solver((n, n, n), "store_some") as a:
        a.step(6)
        full = a.state()
    with solver((n, n, n), "store_some") as b:
        b.step(3)
        mid = b.state()
    with solver((n, n, n), "store_some") as c:
        c.set_state(mid)
        c.step(3)
        resumed = c.state()
    assert np.array_equal(full, resumed)


def test_device_buffers_and_streams():
    n = 16
    st = torch.cuda.Stream()
    ref = O.run(O.tgv_ic(n, n, n, GAMMA, MACH), 2, dt=1e-3)
    with torch.cuda.stream(st):
        with solver((n, n, n), "recompute_all") as s:
            s.step(2)
            out = torch.empty((5, n, n, n), dtype=torch.float64, device="cuda")
            s.state(out)
            R = torch.empty_like(out)
            s.residual(R)
    st.synchronize()
    assert rel_linf(out.cpu().numpy(), ref) <= 1e-12
    assert torch.isfinite(R).all()


def test_cuda_malloc_path_matches_torch_allocator():
    n = 16
    a = fd.Solver(n, dt=1e-3, algorithm="store_all", use_torch_allocator=True)
    b = fd.Solver(n, dt=1e-3, algorithm="store_all", use_torch_allocator=False)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.state(), b.state())
    assert a.device_bytes() == b.device_bytes() > 0
    a.close()
    b.close()


def test_non_finite_state_is_reported():
    n = 8
    with solver((n, n, n), "store_some") as s:
        assert s.check_finite()
        Q = s.state()
        Q[4, 3, 2, 1] = np.nan
        s.set_state(Q)
        assert fd.fd_check_finite(s.h) == fd.FD_EUNSTABLE


def test_bad_sizes_are_rejected():
    n = 8
    with solver((n, n, n), "store_some") as s:
        with pytest.raises(fd.FdError) as e:
            fd.fd_get_state(s.h, np.empty(10))
        assert e.value.code == fd.FD_EINVAL
        with pytest.raises(fd.FdError):
            fd.fd_step(s.h, -1)


@pytest.mark.parametrize("dtype", ["f64", "f32", "df64"])
def test_async_state_copies_match_the_synchronising_calls(dtype):
    """fd_set_state_async / fd_get_state_async through pinned host buffers, with
    two solvers on two streams taking steps in turn, give the same bits as the
    synchronising calls on one solver."""
    from paper_1610_09146_gb300 import native
    shape = (20, 24, 28)
    Q0 = smooth_state(shape, seed=51)
    nel = Q0.size
    with solver(shape, "store_some", dtype=dtype) as s:
        s.set_state(Q0)
        s.step(1)
        want = s.state()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    hin = torch.from_numpy(Q0.reshape(-1).copy()).pin_memory()
    outs = [torch.empty(nel, dtype=torch.float64, pin_memory=True) for _ in streams]
    sols = [fd.Solver(shape[::-1], Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA, dt=1e-3, algorithm="store_some",
                      dtype=dtype, stream=st) for st in streams]
    try:
        for k in range(4):
            sv, o = sols[k % 2], outs[k % 2]
            native.fd_set_state_async(sv.h, hin.data_ptr(), nel, 0)
            native.fd_step(sv.h, 1)
            native.fd_get_state_async(sv.h, o.data_ptr(), nel, 0)
        torch.cuda.synchronize()
        for o in outs:
            assert np.array_equal(o.numpy().reshape(Q0.shape), want)
    finally:
        for sv in sols:
            sv.close()


@pytest.mark.slow
def test_store_all_beyond_32bit_work_array_offsets():
    """At 384^3 the store-all work arrays span 45 n > 2^31 values, so their
    offsets need 64 bits: one BL step against the oracle at sampled points
    (random, and next to every face of the box), as the 256^3 test does."""
    n = 384
    dt = fd.dt_for_grid(n)
    Q0 = O.tgv_ic(n, n, n, GAMMA, MACH)
    rng = np.random.default_rng(384)
    pts = [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(12)]
    pts += [(0, 0, 0), (n - 1, n - 1, n - 1), (n - 1, 0, 191), (0, n - 2, n - 1)]
    ref = oracle_one_step_at(Q0, pts, dt, (2 * np.pi / n,) * 3)
    scale = np.abs(Q0).reshape(5, -1).max(axis=1)
    scale[3] = np.abs(ref[:, 3]).max()
    with solver((n, n, n), "store_all", dt=dt) as s:
        s.step(1)
        Q = s.state()
    got = np.array([Q[:, z, y, x] for (z, y, x) in pts])
    for v in range(5):
        assert np.abs(got[:, v] - ref[:, v]).max() <= 1e-12 * scale[v], v
