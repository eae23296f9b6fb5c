"""Pins for the oracle's low-storage three-stage Runge-Kutta scheme (Section 2, Fig. 1).

The paper says only "low storage ... three stages"; the reading is a
two-register scheme.  These tests fix it by what any 3-stage, 3rd-order
explicit RK must satisfy: the classical order conditions of its Butcher
tableau, the stability polynomial 1 + z + z^2/2 + z^3/6 on linear problems,
and a measured temporal order of 3 on a nonlinear scalar ODE and on the full
Navier-Stokes solver.
"""
import numpy as np
import pytest

import oracle as O


def test_butcher_order_conditions():
    a, b = O.rk_coefficients()
    # two-register scheme Q <- Qs + a_s dt R, Qs <- Qs + b_s dt R, Qs = Q at save-state:
    #   stage 2 input = Q0 + a0 dt k1
    #   stage 3 input = Q0 + b0 dt k1 + a1 dt k2
    #   result        = Q0 + b0 dt k1 + b1 dt k2 + a2 dt k3
    A = np.array([[0, 0, 0], [a[0], 0, 0], [b[0], a[1], 0]])
    w = np.array([b[0], b[1], a[2]])
    c = A.sum(axis=1)
    assert w.sum() == pytest.approx(1, abs=1e-15)
    assert w @ c == pytest.approx(1 / 2, abs=1e-15)
    assert w @ c**2 == pytest.approx(1 / 3, abs=1e-15)
    assert w @ A @ c == pytest.approx(1 / 6, abs=1e-15)


@pytest.mark.parametrize("z", [-0.5, -1.3, 0.2, -2.4])
def test_stability_polynomial_real(z):
    q = O.lsrk3_step(np.array([1.0]), 1.0, lambda q: z * q)
    assert q[0] == pytest.approx(1 + z + z**2 / 2 + z**3 / 6, abs=1e-15)


@pytest.mark.parametrize("zr,zi", [(0.0, 1.0), (-0.3, 1.5), (-1.0, -0.7)])
def test_stability_polynomial_complex(zr, zi):
    A = np.array([[zr, -zi], [zi, zr]])
    q = O.lsrk3_step(np.array([1.0, 0.0]), 1.0, lambda q: A @ q)
    z = complex(zr, zi)
    P = 1 + z + z**2 / 2 + z**3 / 6
    np.testing.assert_allclose(q, [P.real, P.imag], atol=1e-15)


def test_third_order_on_nonlinear_ode():
    # q' = q^2, q(0) = 1  ->  q(t) = 1 / (1 - t)
    errs = []
    for nst in (10, 20, 40):
        dt = 0.4 / nst
        q = np.array([1.0])
        for _ in range(nst):
            q = O.lsrk3_step(q, dt, lambda v: v * v)
        errs.append(abs(q[0] - 1 / (1 - 0.4)))
    p = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(p - 3) < 0.15), p


@pytest.mark.slow
def test_third_order_in_time_on_navier_stokes():
    n, mach, tend = 16, 0.5, 0.2
    Q0 = O.tgv_ic(n, n, n, 1.4, mach)
    ref = O.run(Q0, 160, dt=tend / 160, Mach=mach)
    errs = []
    for nst in (10, 20, 40):
        Q = O.run(Q0, nst, dt=tend / nst, Mach=mach)
        errs.append(np.abs(Q - ref).max())
    p = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(p - 3) < 0.3), (p, errs)
