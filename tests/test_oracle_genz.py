"""Pins for the oracle's Genz 1984 integrands and their closed-form
integrals.  The integrand (or_genz) and the closed form (or_genz_exact) are
separate formulas; each closed form is checked against independent
numerical quadrature of the integrand (scipy's adaptive quad, and a
tensor Gauss-Legendre rule built from numpy's nodes), so a dropped term or
wrong sign on either side fails here."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O

FAMS = [O.OSCILLATORY, O.PRODUCT_PEAK, O.CORNER_PEAK, O.GAUSSIAN, O.C0,
        O.DISCONTINUOUS]


def _params(ndim, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 3.0, ndim), rng.uniform(0.1, 0.9, ndim)


@pytest.mark.parametrize("fam", FAMS)
def test_closed_form_1d_against_adaptive_quadrature(fam):
    a, u = _params(1, 10 + fam)
    f = lambda x: O.genz(fam, a, u, [x])
    val = sum(integrate.quad(f, lo, hi, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
              for lo, hi in [(0.0, u[0]), (u[0], 1.0)])
    assert val == pytest.approx(O.genz_exact(fam, a, u), rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("fam", FAMS)
def test_closed_form_2d_against_adaptive_quadrature(fam):
    a, u = _params(2, 20 + fam)
    f = lambda y, x: O.genz(fam, a, u, [x, y])
    total = 0.0
    for x0, x1 in [(0.0, u[0]), (u[0], 1.0)]:
        for y0, y1 in [(0.0, u[1]), (u[1], 1.0)]:
            total += integrate.dblquad(f, x0, x1, y0, y1, epsabs=1e-13, epsrel=1e-12)[0]
    assert total == pytest.approx(O.genz_exact(fam, a, u), rel=1e-9, abs=1e-12)


@pytest.mark.parametrize("fam", [O.OSCILLATORY, O.PRODUCT_PEAK, O.CORNER_PEAK, O.GAUSSIAN])
def test_closed_form_3d_against_gauss_legendre(fam):
    # smooth families: a 48^3-point tensor Gauss-Legendre rule is exact to
    # far below the tolerance.
    a, u = _params(3, 30 + fam)
    t, w = np.polynomial.legendre.leggauss(48)
    t, w = 0.5 * (t + 1.0), 0.5 * w
    acc = 0.0
    for i, xi in enumerate(t):
        for j, xj in enumerate(t):
            for k, xk in enumerate(t):
                acc += w[i] * w[j] * w[k] * O.genz(fam, a, u, [xi, xj, xk])
    assert acc == pytest.approx(O.genz_exact(fam, a, u), rel=1e-10)


def test_gaussian3d_a5_closed_form():
    # a_i = 5, u_i = 1/2 in 3 dimensions: (sqrt(pi)/5 erf(5/2))^3.
    expect = (math.sqrt(math.pi) / 5.0 * math.erf(2.5)) ** 3
    val = O.genz_exact(O.GAUSSIAN, [5.0] * 3, [0.5] * 3)
    assert val == pytest.approx(expect, rel=1e-15)
    assert val == pytest.approx(0.044492261088252646, rel=1e-15)


@pytest.mark.parametrize("ndim", range(1, 9))
def test_corner_peak_one_dimensional_form_matches_inclusion_exclusion(ndim):
    rng = np.random.default_rng(ndim)
    a = rng.uniform(0.2, 1.5, ndim)
    assert O.genz_exact(O.CORNER_PEAK, a, np.zeros(ndim)) == pytest.approx(
        O.corner_peak_incl_excl(a), rel=1e-11)


def test_corner_peak_1d_closed_form():
    for a in (0.1, 1.0, 7.5):
        assert O.genz_exact(O.CORNER_PEAK, [a], [0.0]) == pytest.approx(1.0 / (1.0 + a), rel=1e-14)


def test_corner_peak_high_dimension_is_stable():
    # 32 dimensions, sum a = 8 (the scaled parameters of the mixed workload):
    # the value stays positive, below 1, and decreases as a grows.
    a = np.full(32, 0.25)
    v1 = O.genz_exact(O.CORNER_PEAK, a, np.zeros(32))
    v2 = O.genz_exact(O.CORNER_PEAK, 2 * a, np.zeros(32))
    assert 0.0 < v2 < v1 < 1.0
    # Monte Carlo cross-check with plain uniform points
    rng = np.random.default_rng(5)
    x = rng.random((200000, 32))
    mc = np.mean((1.0 + x @ a) ** -33.0)
    sd = np.std((1.0 + x @ a) ** -33.0) / math.sqrt(x.shape[0])
    assert abs(mc - v1) < 5 * sd


def test_oscillatory_phase_shift():
    # u_1 shifts the phase by 2 pi u_1; u_1 = 1/4 turns cos into -sin.
    a = np.array([1.3, 0.7])
    v0 = O.genz_exact(O.OSCILLATORY, a, [0.0, 0.0])
    v4 = O.genz_exact(O.OSCILLATORY, a, [0.25, 0.0])
    # integral of cos(s) and -sin(s), s = a.x, done with quad independently
    fc = integrate.dblquad(lambda y, x: math.cos(a[0] * x + a[1] * y), 0, 1, 0, 1)[0]
    fs = integrate.dblquad(lambda y, x: -math.sin(a[0] * x + a[1] * y), 0, 1, 0, 1)[0]
    assert v0 == pytest.approx(fc, rel=1e-12)
    assert v4 == pytest.approx(fs, rel=1e-12)


def test_discontinuous_cuts_only_first_two_axes():
    a = np.array([0.5, 0.5, 0.5])
    u = np.array([0.3, 0.6, 0.1])
    assert O.genz(O.DISCONTINUOUS, a, u, [0.31, 0.1, 0.9]) == 0.0
    assert O.genz(O.DISCONTINUOUS, a, u, [0.1, 0.61, 0.9]) == 0.0
    assert O.genz(O.DISCONTINUOUS, a, u, [0.29, 0.59, 0.9]) == pytest.approx(
        math.exp(0.5 * (0.29 + 0.59 + 0.9)), rel=1e-15)


def test_const_family():
    assert O.genz(O.CONST, [1.0], [0.5], [0.3]) == 1.0
    assert O.genz_exact(O.CONST, [1.0, 2.0], [0.5, 0.5]) == 1.0
