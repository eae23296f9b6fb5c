"""binary32-stencil mode (FD_F32_ACCDW: compensated binary32 state and RK
accumulation, binary64 reductions) against binary64.

Bounds: relative L2 <= 1e-5 per conserved variable and relative kinetic
energy error <= 1e-6 after 100 steps of the 64^3 Taylor-Green vortex, against
the binary64 GPU run, which is itself checked against the oracle at 64^3.
"""
import numpy as np
import pytest

import oracle as O
from tests.inputs import smooth_state

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402

VARIANTS = ["store_all", "store_some", "recompute_all", "recompute_some", "store_none"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


def rel_l2(a, b):
    return max(np.linalg.norm(a[v] - b[v]) / np.linalg.norm(b[v]) for v in range(5))


@pytest.fixture(scope="module")
def f64_64():
    n = 64
    dt = fd.dt_for_grid(n)
    ref10 = O.run(O.tgv_ic(n, n, n, 1.4, 0.1), 10, dt=dt)
    with fd.Solver(n, dt=dt, algorithm="store_some", dtype="f64") as s:
        s.step(10)
        Q10 = s.state()
        s.step(90)
        Q100 = s.state()
        ke = s.diagnostics()[0]
    return dict(dt=dt, ref10=ref10, Q10=Q10, Q100=Q100, ke=ke)


def test_f64_reference_validated_against_oracle_at_64(f64_64):
    ref, Q = f64_64["ref10"], f64_64["Q10"]
    for v in range(5):
        assert np.abs(Q[v] - ref[v]).max() <= 1e-12 * np.abs(ref[v]).max()


@pytest.mark.parametrize("alg", VARIANTS)
def test_mixed_100_steps_within_bounds(alg, f64_64):
    n = 64
    with fd.Solver(n, dt=f64_64["dt"], algorithm=alg, dtype="f32") as s:
        s.step(100)
        Q = s.state()
        ke = s.diagnostics()[0]
    err = rel_l2(Q, f64_64["Q100"])
    kerr = abs(ke - f64_64["ke"]) / f64_64["ke"]
    print(f"{alg}: rel L2 {err:.3e}  KE rel {kerr:.3e}")
    assert err <= 1e-5
    assert kerr <= 1e-6


@pytest.mark.parametrize("alg", VARIANTS)
def test_mixed_residual_close_to_oracle(alg):
    shape = (20, 22, 24)
    Q0 = smooth_state(shape, seed=9)
    ref = O.residual(Q0)
    with fd.Solver(shape[::-1], dt=1e-3, algorithm=alg, dtype="f32") as s:
        s.set_state(Q0)
        R = s.residual()
    for v in range(5):
        assert np.abs(R[v] - ref[v]).max() <= 2e-5 * np.abs(ref[v]).max(), v


def test_mixed_variants_agree():
    n = 32
    out = {}
    for alg in VARIANTS:
        with fd.Solver(n, dt=1e-3, algorithm=alg, dtype="f32") as s:
            s.step(10)
            out[alg] = s.state()
    for alg in VARIANTS[1:]:
        assert rel_l2(out[alg], out["store_all"]) <= 1e-7, alg

