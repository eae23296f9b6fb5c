"""Mixed binary64 / double-word store-some (dtype "f64dw") against the FP64 oracle.

The mode keeps the state, the RK update and the pressure of Eq. 6 in binary64
and evaluates the other residual terms in double-word arithmetic, and it is
held to the binary64 bound of the plain binary64 path: relative L-inf <= 1e-12
per conserved variable (normalised by max|oracle| of that variable) for the
residual, after 10 steps, and after one step of the 256^3 grid at sampled points,
where the smallest variable (rho w, at most 2e-4 after one step) resolves the
binary64 rounding of the pressure.
"""
import numpy as np
import pytest

import oracle as O
from tests.inputs import rough_state, smooth_state
from tests.sampled import oracle_one_step_at

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402

GAMMA, MACH, RE, PR = 1.4, 0.1, 1600.0, 0.71


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


def rel_linf(a, b):
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(5))


def solver(shape, dt=1e-3, dtype="f64dw", alg="store_some"):
    nz, ny, nx = shape
    return fd.Solver((nx, ny, nz), Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA, dt=dt, algorithm=alg, dtype=dtype)


@pytest.mark.parametrize("shape,kind", [((23, 19, 21), "rough"), ((32, 32, 32), "smooth"), ((5, 6, 7), "rough")])
def test_residual_matches_oracle(shape, kind):
    Q0 = rough_state(shape, seed=5) if kind == "rough" else smooth_state(shape, seed=6)
    ref = O.residual(Q0, Re=RE, Mach=MACH, Pr=PR, gamma=GAMMA)
    with solver(shape) as s:
        s.set_state(Q0)
        R = s.residual()
    assert rel_linf(R, ref) <= 1e-12


def test_residual_of_taylor_green_state_matches_oracle():
    n = 48
    Q0 = O.tgv_ic(n, n, n, GAMMA, MACH)
    ref = O.residual(Q0)
    with solver((n, n, n)) as s:
        R = s.residual()
    assert rel_linf(R, ref) <= 1e-12


def test_ten_steps_tgv_32_matches_oracle():
    n = 32
    ref = O.run(O.tgv_ic(n, n, n, GAMMA, MACH), 10, dt=1e-3)
    with solver((n, n, n)) as s:
        s.step(10)
        Q = s.state()
        ke, en = s.diagnostics()
    assert rel_linf(Q, ref) <= 1e-12
    ke_ref, en_ref = O.diagnostics(ref)
    assert abs(ke - ke_ref) <= 1e-13 * ke_ref and abs(en - en_ref) <= 1e-13 * en_ref


@pytest.mark.parametrize("mach", [0.25, 0.4])
def test_higher_mach_taylor_green_matches_oracle(mach):
    """Above Mach ~0.3 the mean pressure p0 = 1/(gamma M^2) is small enough that the
    double-word p - p0 of the working fields may round (to 2^-48 of itself) instead of
    holding the binary64 value exactly; the residual and ten steps still meet the
    binary64 bound."""
    n = 48
    Q0 = O.tgv_ic(n, n, n, GAMMA, mach)
    ref = O.residual(Q0, Re=RE, Mach=mach, Pr=PR, gamma=GAMMA)
    with fd.Solver((n, n, n), Re=RE, Mach=mach, Pr=PR, gamma=GAMMA, dt=1e-3, algorithm="store_some",
                   dtype="f64dw") as s:
        assert rel_linf(s.residual(), ref) <= 1e-12
    m = 32
    ref = O.run(O.tgv_ic(m, m, m, GAMMA, mach), 10, dt=1e-3, Re=RE, Mach=mach, Pr=PR, gamma=GAMMA)
    with fd.Solver((m, m, m), Re=RE, Mach=mach, Pr=PR, gamma=GAMMA, dt=1e-3, algorithm="store_some",
                   dtype="f64dw") as s:
        s.step(10)
        assert rel_linf(s.state(), ref) <= 1e-12


def test_ten_steps_random_ragged_grid_matches_oracle():
    shape = (18, 24, 20)
    Q0 = smooth_state(shape, seed=21)
    ref = O.run(Q0, 10, dt=1e-3)
    with solver(shape) as s:
        s.set_state(Q0)
        s.step(10)
        assert rel_linf(s.state(), ref) <= 1e-12


def test_smallest_grid_and_zero_steps():
    shape = (5, 5, 5)
    Q0 = smooth_state(shape, seed=2)
    ref = O.run(Q0, 3, dt=1e-3)
    with solver(shape) as s:
        s.set_state(Q0)
        s.step(0)
        assert np.array_equal(s.state(), Q0)  # binary64 state: set / get is exact
        s.step(3)
        assert rel_linf(s.state(), ref) <= 1e-12


def test_agrees_with_binary64_path_at_64():
    n = 64
    dt = fd.dt_for_grid(n)
    out = {}
    for dtype in ("f64", "f64dw"):
        with solver((n, n, n), dt=dt, dtype=dtype) as s:
            s.step(20)
            out[dtype] = s.state()
    assert rel_linf(out["f64dw"], out["f64"]) <= 1e-12


def test_other_families_are_rejected():
    for alg in ("store_all", "recompute_all", "recompute_some", "store_none"):
        with pytest.raises(fd.FdError) as e:
            solver((8, 8, 8), alg=alg)
        assert e.value.code == fd.FD_EINVAL


@pytest.mark.slow
def test_full_size_256_one_step_sampled():
    n = 256
    dt = fd.dt_for_grid(n)
    Q0 = O.tgv_ic(n, n, n, GAMMA, MACH)
    rng = np.random.default_rng(256)
    pts = [tuple(rng.integers(0, n, 3)) for _ in range(24)] + [(0, 0, 0), (n - 1, n - 1, n - 1), (1, n - 2, 0)]
    ref = oracle_one_step_at(Q0, pts, dt, (2 * np.pi / n,) * 3)
    scale = np.abs(Q0).reshape(5, -1).max(axis=1)
    scale[3] = np.abs(ref[:, 3]).max()
    with solver((n, n, n), dt=dt) as s:
        s.step(1)
        Q = s.state()
    for v in range(3):  # mass and momentum are conserved at full size
        assert abs(Q[v].sum() - Q0[v].sum()) <= 1e-12 * np.abs(Q0[v]).sum() + 1e-9
    got = np.array([Q[:, z, y, x] for (z, y, x) in pts])
    for v in range(5):
        assert np.abs(got[:, v] - ref[:, v]).max() <= 1e-12 * scale[v], v
