"""Seeded synthetic inputs shared by the oracle and the CUDA-path tests.

This module holds no arithmetic of the method: it only draws random smooth
periodic fields.  Both sides of every parity test take their inputs from here
(or from their own implementation of the Taylor-Green initial condition).
"""
from __future__ import annotations

import numpy as np


def smooth_field(shape, rng, kmax=2, amp=1.0, nmodes=4):
    """Sum of `nmodes` random real Fourier modes with integer wavenumbers |k_i| <= kmax
    on the periodic [0, 2*pi)^3 grid x_i = i*2*pi/n; returns [nz][ny][nx]."""
    nz, ny, nx = shape
    x = np.arange(nx) * (2 * np.pi / nx)
    y = np.arange(ny) * (2 * np.pi / ny)
    z = np.arange(nz) * (2 * np.pi / nz)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = np.zeros(shape)
    for _ in range(nmodes):
        k = rng.integers(-kmax, kmax + 1, size=3)
        a = rng.uniform(-1, 1)
        ph = rng.uniform(0, 2 * np.pi)
        f += a * np.cos(k[0] * X + k[1] * Y + k[2] * Z + ph)
    return amp * f / nmodes


def smooth_state(shape, seed, rho_amp=0.1, mom_amp=0.5, energy=180.0, energy_amp=1.0, kmax=2):
    """Random smooth conservative state Q[5][nz][ny][nx] = (rho, rho u, rho v, rho w, rho E).

    rho = 1 + perturbation, momenta O(mom_amp), rho E = `energy` + perturbation.
    With the default energy (about the Taylor-Green value at Mach 0.1) the pressure
    stays positive for any draw."""
    rng = np.random.default_rng(seed)
    Q = np.empty((5,) + tuple(shape))
    Q[0] = 1.0 + smooth_field(shape, rng, kmax, rho_amp)
    for i in range(3):
        Q[1 + i] = smooth_field(shape, rng, kmax, mom_amp)
    Q[4] = energy + smooth_field(shape, rng, kmax, energy_amp)
    return Q


def rough_state(shape, seed, rho_amp=0.05, mom_amp=0.2, energy=180.0, energy_amp=0.5):
    """Like smooth_state but with independent random values at every point (all
    wavenumbers present): exercises every stencil tap and the ragged tails."""
    rng = np.random.default_rng(seed)
    Q = np.empty((5,) + tuple(shape))
    Q[0] = 1.0 + rho_amp * rng.uniform(-1, 1, shape)
    for i in range(3):
        Q[1 + i] = mom_amp * rng.uniform(-1, 1, shape)
    Q[4] = energy + energy_amp * rng.uniform(-1, 1, shape)
    return Q
