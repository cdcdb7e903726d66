"""Pins of the oracle's Suave (subregion-adaptive Vegas, as read in the
oracle source): what the mathematics fixes, not the oracle itself.

- A constant integrand is never split (its first sample has zero variance).
- The final regions tile the unit cube (volumes sum to 1, every point lies
  in exactly one box).
- A function of one coordinate is only ever split along that axis (the
  refined grids of the other axes stay even).
- Genz closed forms are met within 4 sigma, for one and for several splits
  per round, and the error shrinks with the sample budget.
"""
import math

import numpy as np
import pytest

import oracle as O


def _prob(ndim, fam, a, u, nbins=16):
    return O.Problem(ndim, [fam], np.asarray(a, float).reshape(1, ndim), np.asarray(u, float).reshape(1, ndim),
                     nbins=nbins)


def test_constant_integrand_is_not_split():
    # the root's first sample has J = 1 at every point (uniform grid): zero
    # variance, no split; the final pass samples the refined grid (bin counts
    # of 1000 points are not all equal), so 1 is met to the sampling error
    r = O.suave(_prob(3, O.CONST, [1, 1, 1], [0.5] * 3), epsrel=1e-9, maxeval=20000, nnew=1000)
    assert r.nregions == 1 and r.neval == 2000
    assert abs(r.integral[0] - 1.0) < 1e-4 and r.error[0] < 1e-4


def _tiles(boxes, ndim, rng):
    vol = np.prod(boxes[:, :, 1] - boxes[:, :, 0], axis=1)
    assert abs(vol.sum() - 1.0) < 1e-12
    pts = rng.random((4000, ndim))
    inside = np.all((pts[:, None, :] >= boxes[None, :, :, 0]) & (pts[:, None, :] < boxes[None, :, :, 1]), axis=2)
    assert np.all(inside.sum(axis=1) == 1)


@pytest.mark.parametrize("width", [1, 8])
def test_regions_tile_the_cube_and_closed_form_is_met(width):
    p = _prob(3, O.GAUSSIAN, [6.0, 4.0, 5.0], [0.3, 0.6, 0.5])
    r = O.suave(p, epsrel=2e-4, maxeval=400000, nnew=2000, width=width)
    assert r.nregions > 4
    _tiles(r.boxes, 3, np.random.default_rng(width))
    assert abs(r.integral[0] - p.exact()[0]) < 4 * r.error[0]


def test_splits_follow_the_only_varying_axis():
    # a Gaussian in x_1 alone (a = 0 elsewhere: constant in x_0 and x_2)
    p = _prob(3, O.GAUSSIAN, [0.0, 8.0, 0.0], [0.5, 0.3, 0.5])
    r = O.suave(p, epsrel=1e-5, maxeval=100000, nnew=1000, width=4, flatness=2.0)
    assert r.nregions > 2
    for ax in (0, 2):
        assert np.all(r.boxes[:, ax, 0] == 0.0) and np.all(r.boxes[:, ax, 1] == 1.0)
    exact = O.genz_exact(O.GAUSSIAN, np.array([8.0]), np.array([0.3]))  # the other axes give 1
    assert abs(r.integral[0] - exact) < 4 * r.error[0]


@pytest.mark.parametrize("fam,a,u", [(O.PRODUCT_PEAK, [4.0, 3.0], [0.4, 0.7]),
                                     (O.CORNER_PEAK, [2.0, 1.0], [0.5, 0.5])])
def test_other_families_meet_the_closed_form(fam, a, u):
    p = _prob(2, fam, a, u)
    r = O.suave(p, epsrel=1e-4, maxeval=300000, nnew=2000, width=4)
    assert abs(r.integral[0] - p.exact()[0]) < 4 * r.error[0]


def test_discontinuous_family_with_independent_points():
    # the final pass is independent of the partition only for independent
    # points (with one Sobol stream the final points are correlated with the
    # samples that chose the partition)
    p = _prob(2, O.DISCONTINUOUS, [1.0, 2.0], [0.3, 0.6])
    p.gen, p.seed = O.PSEUDO, 1
    r = O.suave(p, epsrel=1e-4, maxeval=300000, nnew=2000, width=4)
    assert abs(r.integral[0] - p.exact()[0]) < 4 * r.error[0]


def test_error_shrinks_with_budget():
    p = _prob(3, O.GAUSSIAN, [6.0, 4.0, 5.0], [0.3, 0.6, 0.5])
    e = [O.suave(p, maxeval=m, nnew=1000, width=2).error[0] for m in (20000, 200000)]
    assert e[1] < 0.5 * e[0]


def test_budget_stop_reports_fail():
    p = _prob(3, O.GAUSSIAN, [6.0, 4.0, 5.0], [0.3, 0.6, 0.5])
    r = O.suave(p, epsrel=1e-9, maxeval=15000, nnew=1000)
    assert r.fail == 1 and r.neval <= 15000
