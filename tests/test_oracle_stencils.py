"""Pins for the oracle's fourth-order central difference operators (Section 2).

The paper names the scheme only ("fourth-order central"); these tests fix what
that means independently of the oracle's code:
  * exactness on polynomials (degree <= 4 for D, <= 5 for D2) at points whose
    stencil does not wrap;
  * the closed-form Fourier symbols of the 5-point operators on periodic modes,
    i*kappa1(k) and -kappa2(k);
  * the measured order of accuracy on smooth fields (4);
  * agreement with an FFT application of those symbols on random fields
    (a second algorithm for the same circulant operator).
"""
import numpy as np
import pytest

import oracle as O


def kappa1(k, h):
    return (8 * np.sin(k * h) - np.sin(2 * k * h)) / (6 * h)


def kappa2(k, h):
    return (30 - 32 * np.cos(k * h) + 2 * np.cos(2 * k * h)) / (12 * h * h)


def _line_field(values, axis, other=3):
    """Embed a 1-D line of values along `axis` in a [z][y][x] array."""
    n = len(values)
    shape = [other, other, other]
    shape[2 - axis] = n
    f = np.empty(shape)
    idx = [slice(None)] * 3
    view = np.moveaxis(f, 2 - axis, -1)
    view[...] = values
    return f


def _line_out(f, axis):
    return np.moveaxis(f, 2 - axis, -1)[0, 0]


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4])
def test_d1_exact_on_polynomials(axis, deg):
    n = 20
    h = 0.1
    x = 0.3 + h * np.arange(n)
    f = _line_field(x**deg, axis)
    d = _line_out(O.d1(f, axis, h), axis)
    exact = deg * x ** (deg - 1) if deg > 0 else 0 * x
    interior = slice(2, n - 2)
    np.testing.assert_allclose(d[interior], exact[interior], rtol=1e-11, atol=1e-11)


def test_d1_not_exact_on_degree5():
    n, h = 20, 0.1
    x = 0.3 + h * np.arange(n)
    d = _line_out(O.d1(_line_field(x**5, 0), 0, h), 0)
    err = np.abs(d[2:-2] - 5 * x[2:-2] ** 4).max()
    # leading error of the 4th-order stencil is -h^4/30 f^(5) = -h^4 * 4
    assert err == pytest.approx(4 * h**4, rel=1e-6)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("deg", [0, 1, 2, 3, 4, 5])
def test_d2_exact_on_polynomials(axis, deg):
    n = 20
    h = 0.1
    x = 0.3 + h * np.arange(n)
    f = _line_field(x**deg, axis)
    d = _line_out(O.d2(f, axis, h), axis)
    exact = deg * (deg - 1) * x ** (deg - 2) if deg > 1 else 0 * x
    interior = slice(2, n - 2)
    np.testing.assert_allclose(d[interior], exact[interior], rtol=1e-9, atol=1e-8)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("k", [1, 3, 7])
def test_fourier_symbols(axis, k):
    n = 16
    h = 2 * np.pi / n
    x = h * np.arange(n)
    ph = 0.37
    f = _line_field(np.sin(k * x + ph), axis)
    d = _line_out(O.d1(f, axis), axis)
    dd = _line_out(O.d2(f, axis), axis)
    np.testing.assert_allclose(d, kappa1(k, h) * np.cos(k * x + ph), atol=1e-13)
    np.testing.assert_allclose(dd, -kappa2(k, h) * np.sin(k * x + ph), atol=1e-12)


def _fft_apply(f, axis, symbol):
    ax = 2 - axis
    n = f.shape[ax]
    h = 2 * np.pi / n
    k = np.fft.fftfreq(n, d=1.0 / n)
    shape = [1, 1, 1]
    shape[ax] = n
    s = symbol(k, h).reshape(shape)
    return np.real(np.fft.ifft(np.fft.fft(f, axis=ax) * s, axis=ax))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_circulant_operators_match_fft(axis):
    rng = np.random.default_rng(7)
    f = rng.standard_normal((12, 10, 14))
    d = O.d1(f, axis)
    dd = O.d2(f, axis)
    np.testing.assert_allclose(d, _fft_apply(f, axis, lambda k, h: 1j * kappa1(k, h)), atol=1e-12)
    np.testing.assert_allclose(dd, _fft_apply(f, axis, lambda k, h: -kappa2(k, h)), atol=1e-11)


def test_fourth_order_convergence():
    errs1, errs2 = [], []
    ns = [32, 64, 128, 256]
    for n in ns:
        h = 2 * np.pi / n
        x = h * np.arange(n)
        f = _line_field(np.exp(np.sin(x)), 0, other=1)
        d = _line_out(O.d1(f, 0), 0)
        dd = _line_out(O.d2(f, 0), 0)
        ex1 = np.cos(x) * np.exp(np.sin(x))
        ex2 = (np.cos(x) ** 2 - np.sin(x)) * np.exp(np.sin(x))
        errs1.append(np.abs(d - ex1).max())
        errs2.append(np.abs(dd - ex2).max())
    p1 = np.log2(np.array(errs1[:-1]) / np.array(errs1[1:]))
    p2 = np.log2(np.array(errs2[:-1]) / np.array(errs2[1:]))
    assert np.all(np.abs(p1[1:] - 4) < 0.05), p1
    assert np.all(np.abs(p2[1:] - 4) < 0.05), p2
