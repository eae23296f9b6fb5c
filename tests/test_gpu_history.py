"""Kinetic-energy and enstrophy histories of the Taylor-Green vortex (Section 3, Fig. 3).

1. The history the library samples (Solver.history, the loop of bench.py's history
   workload) matches the oracle's, sample by sample: 300 RK3 steps of the 32^3 grid,
   kinetic energy and enstrophy every 30 steps, relative error <= 1e-12.
2. The energy budget of the compressible equations closes on the GPU's own states.
   For the periodic cube, with mu = 1/Re and angle brackets volume means,
       -dKE/dt = mu <|omega|^2> + (4/3) mu <(div u)^2> - <p' div u>,
   so the density-weighted enstrophy Omega of the diagnostics gives
       -dKE/dt - 2 nu Omega = 2 nu <(1 - rho)|omega|^2/2> + (4/3) nu <(div u)^2> - <p' div u>.
   At Mach 0.1 the pressure-dilatation term oscillates (acoustic waves) at a few
   per cent of the dissipation, so -dKE/dt and 2 nu Omega alone differ by up to
   ~4 % (checked as such), while the full budget closes to the error of the
   central time difference of KE: A w^2 dt_s^2 / 6 with the acoustic amplitude
   A <= 0.04 eps, w <= c |k| = (1/M) 2 sqrt(2) for the TGV pressure modes and
   dt_s = 5 steps, i.e. <= 1.5e-3 eps, plus the fourth-order truncation of the
   derivatives (~(k h)^4 / 30 < 1e-4 at 64^3); the bound used is 2e-3.
   The right-hand side is evaluated here with numpy fourth-order differences of
   the GPU state (test code, independent of the library and of the oracle).
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1610_09146_gb300 as fd  # noqa: E402

GAMMA, MACH, RE = 1.4, 0.1, 1600.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    fd.build()


@pytest.mark.parametrize("dtype", ["f64", "f64dw"])
def test_history_32_matches_oracle(dtype):
    n, per, samples = 32, 30, 10
    dt = fd.dt_for_grid(n)
    with fd.Solver(n, dt=dt, algorithm="store_some", dtype=dtype) as s:
        t, ke, en = s.history(per, samples)
        Q = s.state()
    Qo = O.tgv_ic(n, n, n, GAMMA, MACH)
    for i in range(samples + 1):
        if i:
            Qo = O.run(Qo, per, dt=dt)
        ke_o, en_o = O.diagnostics(Qo)
        assert abs(t[i] - i * per * dt) < 1e-12
        assert abs(ke[i] - ke_o) <= 1e-12 * ke_o, (i, ke[i], ke_o)
        assert abs(en[i] - en_o) <= 1e-12 * en_o, (i, en[i], en_o)
    err = max(np.abs(Q[v] - Qo[v]).max() / np.abs(Qo[v]).max() for v in range(5))
    assert err <= 1e-12


def _budget_terms(Q, h):
    """<|omega|^2/2>, <rho |omega|^2/2>, <(div u)^2>, <p' div u> with 4th-order differences."""

    def d(f, ax):
        return (8 * (np.roll(f, -1, ax) - np.roll(f, 1, ax)) - (np.roll(f, -2, ax) - np.roll(f, 2, ax))) / (12 * h)

    rho = Q[0]
    u, v, w = Q[1] / rho, Q[2] / rho, Q[3] / rho
    p = (GAMMA - 1) * (Q[4] - 0.5 * rho * (u * u + v * v + w * w))
    ux, uy, uz = d(u, 2), d(u, 1), d(u, 0)
    vx, vy, vz = d(v, 2), d(v, 1), d(v, 0)
    wx, wy, wz = d(w, 2), d(w, 1), d(w, 0)
    om2 = (wy - vz) ** 2 + (uz - wx) ** 2 + (vx - uy) ** 2
    div = ux + vy + wz
    return (np.mean(0.5 * om2), np.mean(0.5 * rho * om2), np.mean(div**2), np.mean((p - p.mean()) * div))


def test_energy_budget_closes_at_64():
    n, per, samples = 64, 5, 24
    dt = fd.dt_for_grid(n)
    h = 2 * np.pi / n
    nu = 1.0 / RE
    ke, omega, terms = [], [], []
    with fd.Solver(n, dt=dt, algorithm="store_some", dtype="f64dw") as s:
        for i in range(samples + 1):
            if i:
                s.step(per)
            k, e = s.diagnostics()
            ke.append(k)
            omega.append(e)
            terms.append(_budget_terms(s.state(), h))
    ke = np.array(ke)
    dts = per * dt
    worst_full, worst_plain = 0.0, 0.0
    for i in range(1, samples):
        eps = -(ke[i + 1] - ke[i - 1]) / (2 * dts)
        ens_u, ens_rho, div2, pdil = terms[i]
        assert abs(ens_rho - omega[i]) <= 1e-12 * omega[i]  # the library's enstrophy is <rho |omega|^2 / 2>
        rhs = 2 * nu * ens_u + (4.0 / 3.0) * nu * div2 - pdil
        worst_full = max(worst_full, abs(eps - rhs) / eps)
        worst_plain = max(worst_plain, abs(eps - 2 * nu * omega[i]) / eps)
    assert worst_full <= 2e-3, worst_full
    assert worst_plain <= 5e-2, worst_plain
