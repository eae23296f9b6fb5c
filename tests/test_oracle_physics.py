"""Pins for the oracle's residual, initial condition and diagnostics.

Each test checks the oracle against something fixed by the paper or by
mathematics, never against itself:
  * closed forms of the Taylor-Green initial state (Section 3, DeBonis 2013):
    mean kinetic energy 1/8, the discrete enstrophy, T = 1, zero divergence;
  * special states in which the residual of Eqs. 1-5 reduces to a closed form
    of the 5-point operators' Fourier symbols (pure heat conduction, Galilean
    advection, linear viscous diffusion);
  * consistency with the continuous equations 1-7 differentiated exactly
    (sympy), converging at 4th order;
  * discrete conservation of mass and momentum on the periodic grid;
  * the reflection and swap symmetries of the Taylor-Green flow.
"""
import numpy as np
import pytest

import oracle as O
from tests.inputs import smooth_state

GAMMA = 1.4


def kappa1(k, h):
    return (8 * np.sin(k * h) - np.sin(2 * k * h)) / (6 * h)


def kappa2(k, h):
    return (30 - 32 * np.cos(k * h) + 2 * np.cos(2 * k * h)) / (12 * h * h)


def grid(n):
    x = np.arange(n) * (2 * np.pi / n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


# ---------------------------------------------------------------- Section 3 IC


@pytest.mark.parametrize("n", [8, 16, 32])
@pytest.mark.parametrize("mach", [0.1, 0.4])
def test_tgv_initial_kinetic_energy_is_one_eighth(n, mach):
    ke, _ = O.diagnostics(O.tgv_ic(n, n, n, GAMMA, mach))
    assert abs(ke - 0.125) < 1e-15


@pytest.mark.parametrize("n", [8, 16, 32])
@pytest.mark.parametrize("mach", [0.1, 0.4])
def test_tgv_initial_enstrophy_closed_form(n, mach):
    # With the 4th-order curl, omega = kappa1(1) * (continuous omega) and the
    # density weighting contributes -5 gamma M^2/128 (hand-derived from the IC).
    h = 2 * np.pi / n
    _, ens = O.diagnostics(O.tgv_ic(n, n, n, GAMMA, mach))
    expect = kappa1(1, h) ** 2 * (3.0 / 8.0 - 5.0 * GAMMA * mach**2 / 128.0)
    assert abs(ens - expect) < 1e-15


@pytest.mark.parametrize("n", [8, 12, 16])
def test_kinetic_energy_is_density_weighted(n):
    # rho = 1 + a cos 2x, u = sin x: <rho u^2 / 2> = (1/2 - a/4) / 2 on any grid of
    # more than 4 points (the unweighted mean would be 1/4)
    a = 0.3
    X, Y, Z = grid(n)
    rho = 1.0 + a * np.cos(2 * X)
    Q = np.zeros((5, n, n, n))
    Q[0] = rho
    Q[1] = rho * np.sin(X)
    Q[4] = 200.0
    ke, _ = O.diagnostics(Q)
    assert abs(ke - (0.25 - a / 8)) < 1e-15


@pytest.mark.parametrize("n", [8, 16])
def test_curl_free_field_has_zero_enstrophy(n):
    # u = v = w = f(x + y + z) on a cubic grid: every D_j u_i differences the same
    # stencil values (up to the rounding of x + y + z), so each vorticity component
    # is a difference of two equal numbers; a sign slip would give |omega| ~ 1
    X, Y, Z = grid(n)
    f = 0.5 * np.sin(X + Y + Z)
    rho = 1.0 + 0.1 * np.cos(2 * X)
    Q = np.zeros((5, n, n, n))
    Q[0] = rho
    Q[1] = Q[2] = Q[3] = rho * f
    Q[4] = 200.0
    ke, ens = O.diagnostics(Q)
    assert ens < 1e-24
    assert abs(ke - 0.1875) < 1e-15  # 3/2 <rho f^2>, the cos 2x weighting averages out here


def test_tgv_initial_state_fields():
    n = 16
    Q = O.tgv_ic(n, n, n, GAMMA, 0.1)
    X, Y, Z = grid(n)
    prim = O.primitives(Q, GAMMA, 0.1)
    np.testing.assert_allclose(prim[0], np.sin(X) * np.cos(Y) * np.cos(Z), atol=1e-15)
    np.testing.assert_allclose(prim[1], -np.cos(X) * np.sin(Y) * np.cos(Z), atol=1e-15)
    np.testing.assert_allclose(prim[2], 0.0, atol=0)
    np.testing.assert_allclose(prim[4], 1.0, atol=1e-14)  # T = gamma M^2 p / rho = 1
    div = O.d1(prim[0], 0) + O.d1(prim[1], 1) + O.d1(prim[2], 2)
    assert np.abs(div).max() < 1e-14


# ------------------------------------------ residual: closed-form special states


def test_pure_heat_conduction_state():
    """u = 0, rho = 1: the residual of Eqs. 1-3 is R_rho = 0, R_rhou_i = -D_i p,
    R_rhoE = kappa_T sum_j D2_j T with T = gamma M^2 p (Eq. 5 and Eq. 7)."""
    n, mach, Re, Pr = 16, 0.1, 1600.0, 0.71
    h = 2 * np.pi / n
    X, Y, Z = grid(n)
    k = np.array([1, -2, 3])
    th = k[0] * X + k[1] * Y + k[2] * Z + 0.4
    p0, eps = 1 / (GAMMA * mach**2), 0.5
    p = p0 + eps * np.cos(th)
    Q = np.zeros((5, n, n, n))
    Q[0] = 1.0
    Q[4] = p / (GAMMA - 1)
    R = O.residual(Q, Re=Re, Mach=mach, Pr=Pr, gamma=GAMMA)
    kap = 1 / ((GAMMA - 1) * mach**2 * Pr * Re)
    assert np.abs(R[0]).max() == 0.0
    for i in range(3):
        np.testing.assert_allclose(R[1 + i], eps * kappa1(k[i], h) * np.sin(th), atol=1e-12)
    lapT = -GAMMA * mach**2 * eps * sum(kappa2(kk, h) for kk in k) * np.cos(th)
    np.testing.assert_allclose(R[4], kap * lapT, atol=1e-12, rtol=0)
    assert np.abs(kap * lapT).max() > 1e-3


def test_galilean_advection_state():
    """Uniform velocity U and pressure, rho = 1 + eps cos(k.x), no diffusion:
    R_rho = -U_j D_j rho, R_rhou_i = U_i R_rho, R_rhoE = |U|^2/2 R_rho
    (Eqs. 1-3 with the skew form reduce to pure advection)."""
    n, mach = 16, 0.5
    h = 2 * np.pi / n
    X, Y, Z = grid(n)
    k = np.array([2, 1, -1])
    th = k[0] * X + k[1] * Y + k[2] * Z + 1.1
    eps = 0.2
    U = np.array([0.7, -0.4, 0.25])
    rho = 1 + eps * np.cos(th)
    p0 = 1 / (GAMMA * mach**2)
    Q = np.empty((5, n, n, n))
    Q[0] = rho
    for i in range(3):
        Q[1 + i] = rho * U[i]
    Q[4] = p0 / (GAMMA - 1) + 0.5 * rho * (U @ U)
    R = O.residual(Q, Re=1e30, Mach=mach, Pr=0.71, gamma=GAMMA)
    Rrho = eps * sum(U[j] * kappa1(k[j], h) for j in range(3)) * np.sin(th)
    np.testing.assert_allclose(R[0], Rrho, atol=1e-12)
    for i in range(3):
        np.testing.assert_allclose(R[1 + i], U[i] * Rrho, atol=1e-11)
    np.testing.assert_allclose(R[4], 0.5 * (U @ U) * Rrho, atol=1e-11)


def test_linear_viscous_state():
    """rho = 1, uniform p, velocity a tiny single Fourier mode with nonzero
    divergence, Re = 1: to first order in the amplitude the momentum residual
    is the expanded viscous term (Eq. 4) with the pure second derivative
    symbol for D_jj and kappa1*kappa1 for the mixed D_i D_k (i != k), and the
    mass residual is -D_j u_j, the energy residual the enthalpy flux
    -(rho E + p) D_j u_j = -gamma p0/(gamma-1) D_j u_j."""
    n, mach, Re = 16, 1.0, 1.0
    h = 2 * np.pi / n
    X, Y, Z = grid(n)
    k = np.array([3, -1, 2])
    th = k[0] * X + k[1] * Y + k[2] * Z
    eps = 1e-6
    C = np.array([1.0, -0.6, 0.8])
    ph = np.array([0.3, 1.7, -0.9])
    u = [eps * C[i] * np.sin(th + ph[i]) for i in range(3)]
    p0 = 1 / (GAMMA * mach**2)
    Q = np.empty((5, n, n, n))
    Q[0] = 1.0
    for i in range(3):
        Q[1 + i] = u[i]
    Q[4] = p0 / (GAMMA - 1) + 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    R = O.residual(Q, Re=Re, Mach=mach, Pr=0.71, gamma=GAMMA)
    lap = -sum(kappa2(kk, h) for kk in k)
    for i in range(3):
        mixed = -kappa2(k[i], h) * u[i]
        for kk in range(3):
            if kk != i:
                mixed = mixed - eps * C[kk] * kappa1(k[kk], h) * kappa1(k[i], h) * np.sin(th + ph[kk])
        expect = (1 / Re) * (lap * u[i] + mixed / 3)
        scale = np.abs(expect).max()
        assert np.abs(R[1 + i] - expect).max() < 1e-5 * scale
    div = sum(eps * C[j] * kappa1(k[j], h) * np.cos(th + ph[j]) for j in range(3))
    np.testing.assert_allclose(R[0], -div, atol=1e-9 * np.abs(div).max())
    enth = -GAMMA * p0 / (GAMMA - 1) * div
    assert np.abs(R[4] - enth).max() < 1e-5 * np.abs(enth).max()


# ------------------------------------- consistency with the continuous Eqs. 1-7


def _exact_rhs(n, gamma, mach, Re, Pr):
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    X = (x, y, z)
    rho = 1 + sp.Rational(1, 5) * sp.sin(x) * sp.cos(y) + sp.Rational(1, 10) * sp.cos(z + 0.3)
    u = [sp.Rational(1, 2) * sp.sin(x + 0.1) * sp.cos(y) + sp.Rational(1, 5) * sp.cos(z),
         -sp.Rational(3, 10) * sp.cos(x) * sp.sin(y + 0.2) + sp.Rational(1, 10) * sp.sin(z),
         sp.Rational(2, 5) * sp.sin(z) * sp.cos(x + 0.4) + sp.Rational(1, 10) * sp.cos(y)]
    p0 = 1 / (gamma * mach**2)
    p = p0 + sp.Rational(3, 10) * sp.cos(x - y) + sp.Rational(1, 5) * sp.sin(z)
    rhoE = p / (gamma - 1) + rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2) / 2
    T = gamma * mach**2 * p / rho
    divu = sum(sp.diff(u[k], X[k]) for k in range(3))
    tau = [[(sp.diff(u[i], X[j]) + sp.diff(u[j], X[i])
             - (sp.Rational(2, 3) * divu if i == j else 0)) / Re for j in range(3)] for i in range(3)]
    q = [sp.diff(T, X[j]) / ((gamma - 1) * mach**2 * Pr * Re) for j in range(3)]
    R = [-sum(sp.diff(rho * u[j], X[j]) for j in range(3))]
    for i in range(3):
        R.append(-sum(sp.diff(rho * u[i] * u[j] + (p if i == j else 0) - tau[i][j], X[j])
                      for j in range(3)))
    R.append(-sum(sp.diff(rhoE * u[j] + u[j] * p - q[j] - sum(u[i] * tau[i][j] for i in range(3)), X[j])
                  for j in range(3)))
    cons = [rho, rho * u[0], rho * u[1], rho * u[2], rhoE]
    f_cons = sp.lambdify(X, cons, "numpy")
    f_R = sp.lambdify(X, R, "numpy")
    return f_cons, f_R


@pytest.mark.slow
def test_residual_consistent_with_continuous_equations():
    gamma, mach, Re, Pr = 1.4, 0.5, 50.0, 0.71
    f_cons, f_R = _exact_rhs(None, gamma, mach, Re, Pr)
    errs = []
    for n in (16, 32, 64):
        X, Y, Z = grid(n)
        Q = np.array([np.broadcast_to(c, X.shape) for c in f_cons(X, Y, Z)], dtype=np.float64)
        Rex = np.array([np.broadcast_to(c, X.shape) for c in f_R(X, Y, Z)], dtype=np.float64)
        R = O.residual(Q, Re=Re, Mach=mach, Pr=Pr, gamma=gamma)
        errs.append([np.abs(R[v] - Rex[v]).max() / np.abs(Rex[v]).max() for v in range(5)])
    errs = np.array(errs)
    order = np.log2(errs[1] / errs[2])
    assert np.all(errs[2] < 1e-4), errs
    assert np.all(order > 3.7) and np.all(order < 4.3), (order, errs)


# --------------------------------------------------- conservation and symmetry


def test_mass_and_momentum_conserved():
    n = 16
    Q0 = smooth_state((n, n, n), seed=11)
    Q = O.run(Q0, 40, dt=2e-3)
    assert np.abs(Q - Q0).max() > 1e-3  # the state did evolve
    for v in range(4):
        drift = abs(Q[v].sum() - Q0[v].sum())
        assert drift < 1e-12 * np.abs(Q0[v]).sum(), (v, drift)
    # total energy is not conserved discretely: the viscous work is in product-rule form
    assert abs(Q[4].sum() - Q0[4].sum()) > 1e-12 * np.abs(Q0[4]).sum()


def _reflect(Q, axis):
    n = Q.shape[-1]
    idx = (-np.arange(n)) % n
    ax = 3 - axis
    R = np.take(Q, idx, axis=ax)
    R[1 + axis] *= -1
    return R


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_tgv_reflection_symmetry_preserved(axis):
    n = 16
    Q = O.run(O.tgv_ic(n, n, n, GAMMA, 0.1), 5, dt=5e-3)
    np.testing.assert_allclose(_reflect(Q, axis), Q, atol=1e-12, rtol=0)


def _swap_shift(Q):
    """Reflection x <-> y composed with a shift of pi in x: maps the TGV state to itself."""
    n = Q.shape[-1]
    out = np.swapaxes(np.roll(Q, -n // 2, axis=3), 2, 3).copy()
    out[[1, 2]] = out[[2, 1]]
    return out


def test_tgv_swap_shift_symmetry_preserved():
    n = 16
    Q0 = O.tgv_ic(n, n, n, GAMMA, 0.1)
    np.testing.assert_allclose(_swap_shift(Q0), Q0, atol=1e-14)
    Q = O.run(Q0, 5, dt=5e-3)
    np.testing.assert_allclose(_swap_shift(Q), Q, atol=1e-12, rtol=0)
    # a state without the symmetry is moved by the map (the check has teeth)
    S = smooth_state((n, n, n), seed=3)
    assert np.abs(_swap_shift(S) - S).max() > 1e-2
