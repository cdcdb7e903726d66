"""Pins for the oracle's grid map, sampling pass, refinement, combination
and Vegas driver (Lepage 1978 for the algorithm; the paper gives only the
Vegas argument list, Sect. 3.2.2, and the sampling unit, Sect. 2.1).

Each check uses a property the mathematics fixes: exact sums for f = 1,
exact per-bin counts from the Sobol (0,1)-property, histogram totals equal
to the second moment, integral preservation of the grid map (midpoint
lattice), equal-share rebinning, symmetry and scale invariance of the
refinement, closed-form chi-square probabilities, and 3-sigma agreement of
full runs with Genz closed forms."""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle as O


def _problem(ndim, fams, a, u, nbins=64, bits=52):
    fams = list(fams)
    a = np.broadcast_to(np.asarray(a, float), (len(fams), ndim)).copy()
    u = np.broadcast_to(np.asarray(u, float), (len(fams), ndim)).copy()
    return O.Problem(ndim, fams, a, u, nbins=nbins, bits=bits)


def _random_grid(ndim, nbins, seed):
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.2, 1.0, (ndim, nbins))
    c = np.concatenate([np.zeros((ndim, 1)), np.cumsum(w, axis=1)], axis=1)
    e = c / c[:, -1:]
    e[:, 0], e[:, -1] = 0.0, 1.0
    return e


# ---------------------------------------------------------------- grid map
@pytest.mark.parametrize("nbins", [2, 50, 64, 256])
def test_uniform_grid_partitions_unit_interval(nbins):
    e = O.grid_uniform(3, nbins)
    assert np.all(np.diff(e, axis=1) > 0)
    assert np.all(e[:, 0] == 0.0) and np.all(e[:, -1] == 1.0)
    assert np.all(np.abs(np.diff(e, axis=1).sum(axis=1) - 1.0) <= 2.3e-16)


@pytest.mark.parametrize("bits", [52, 23])
def test_map_of_bin_edges_and_jacobian(bits):
    # y = k/N maps to e_k with J = N w_k per axis.
    e = _random_grid(2, 4, 1)
    for k in range(4):
        Y = np.array([(k << bits) // 4, (k << bits) // 4], dtype=np.uint64)
        x, J, kk = O.map_point(e, Y, bits)
        assert list(kk) == [k, k]
        assert np.array_equal(x, e[:, k])
        assert J == pytest.approx(np.prod(4 * (e[:, k + 1] - e[:, k])), rel=1e-15)


@pytest.mark.parametrize("fam", [O.GAUSSIAN, O.PRODUCT_PEAK, O.OSCILLATORY, O.C0])
def test_grid_map_preserves_integrals_midpoint_lattice(fam):
    # int f(x(y)) J(y) dy over [0,1]^2 = int f(x) dx for any grid: midpoint
    # rule on a 2^8 x 2^8 lattice aligned with the y-bins of a random N = 4
    # grid.
    bits, L = 52, 256
    e = _random_grid(2, 4, 7)
    a, u = np.array([2.0, 3.0]), np.array([0.4, 0.7])
    acc = 0.0
    for i in range(L):
        for j in range(L):
            Y = np.array([(2 * i + 1) << (bits - 9), (2 * j + 1) << (bits - 9)], dtype=np.uint64)
            x, J, _ = O.map_point(e, Y, bits)
            acc += O.genz(fam, a, u, x) * J
    acc /= L * L
    assert acc == pytest.approx(O.genz_exact(fam, a, u), rel=2e-4)


# ---------------------------------------------------------------- sampling
@pytest.mark.parametrize("bits", [52, 23])
def test_constant_integrand_sums_and_counts_exact(bits):
    # f = 1 on a uniform power-of-two grid: J = 1 exactly, S1 = S2 = n, and
    # an aligned block of n = c N points puts exactly c points in every bin of
    # every axis (the (0,1)-property of each Sobol coordinate).
    N, n = 64, 2 ** 14
    p = _problem(5, [O.CONST], 1.0, 0.5, nbins=N, bits=bits)
    S1, S2, H = O.sample(p, O.grid_uniform(5, N), start=3 * n, n=n)
    assert S1[0] == n and S2[0] == n
    assert np.all(H == n // N)


def test_counts_for_non_power_of_two_bins_are_balanced():
    # N = 50: each bin of width 1/50 holds n/50 points up to the (0,1)-
    # sequence discrepancy, a few points at most.
    N, n = 50, 20000
    p = _problem(3, [O.CONST], 1.0, 0.5, nbins=N)
    _, _, H = O.sample(p, O.grid_uniform(3, N), start=1, n=n)
    assert np.all(np.abs(H - n / N) <= 1 + math.log2(n))
    assert np.all(H.sum(axis=1) == n)


def test_histogram_rows_sum_to_second_moment_of_component0():
    p = _problem(4, [O.GAUSSIAN, O.C0], [2.0, 1.0, 3.0, 0.5], [0.3, 0.6, 0.5, 0.2], nbins=32)
    e = _random_grid(4, 32, 3)
    S1, S2, H = O.sample(p, e, start=1, n=5000)
    for d in range(4):
        assert H[d].sum() == pytest.approx(S2[0], rel=1e-13)


def test_bins_agree_with_y_coordinates():
    # with f = 1 the histogram counts how many y fall in each y-bin; the
    # same counts follow from the generated coordinates directly.
    N, n, bits = 50, 3000, 52
    p = _problem(3, [O.CONST], 1.0, 0.5, nbins=N)
    _, _, H = O.sample(p, O.grid_uniform(3, N), start=17, n=n)
    Y = O.sobol_coords(3, 17, n, bits)
    y = Y.astype(np.float64) / 2.0 ** bits
    # (N = 50 widths are not exact in binary, so (J f)^2 = 1 only to rounding)
    for d in range(3):
        np.testing.assert_allclose(
            H[d], np.bincount(np.floor(y[d] * N).astype(int), minlength=N), rtol=1e-12)


def test_estimate_on_random_grid_converges_to_closed_form():
    a, u = [3.0, 2.0, 4.0], [0.4, 0.55, 0.3]
    p = _problem(3, [O.GAUSSIAN], a, u, nbins=16)
    e = _random_grid(3, 16, 11)
    n = 2 ** 16
    S1, S2, _ = O.sample(p, e, start=1, n=n)
    I, var = O.iteration_result(S1, S2, n)
    assert abs(I[0] - p.exact()[0]) < 3 * math.sqrt(var[0])
    assert I[0] == pytest.approx(p.exact()[0], rel=2e-3)


def test_thread_split_is_sum_invariant():
    p = _problem(6, [O.OSCILLATORY, O.PRODUCT_PEAK], 1.5, 0.4, nbins=32)
    e = _random_grid(6, 32, 5)
    r1 = O.sample(p, e, start=5, n=9001, nthreads=1)
    r4 = O.sample(p, e, start=5, n=9001, nthreads=4)
    for x1, x4 in zip(r1, r4):
        np.testing.assert_allclose(x1, x4, rtol=1e-14, atol=1e-300)


def _scipy_points(ndim, start, n):
    # scipy's unscrambled Sobol points at 23 bits (a library special case of
    # the oracle's generator, pinned in test_oracle_sobol.py)
    eng = stats.qmc.Sobol(ndim, scramble=False, bits=52)
    pts = eng.random_base2(int(math.ceil(math.log2(start + n))))[start:start + n]
    return np.floor(pts * 2.0 ** 23) / 2.0 ** 23


@pytest.mark.parametrize("j0", [5, 17, 40])
def test_boundary_mass_counts_exactly_the_points_in_the_band(j0):
    # Discontinuous family on the uniform power-of-two grid (J = 1, x = y).
    # The cut u_1 is put at point j0's own coordinate, u_2 = 1 (never cuts):
    # the only point within the band is j0, and its boundary mass is the
    # value it would have inside, exp(sum a x).  Fixed by the definition of
    # the band, checked against scipy's points.
    ndim, N, start, n = 3, 64, 1, 64
    a = np.array([0.7, 1.1, 0.4])
    y = _scipy_points(ndim, start, n)
    u = np.array([y[j0, 0], 1.0, 0.5])
    p = _problem(ndim, [O.DISCONTINUOUS], a, u, nbins=N, bits=23)
    r = O.sample_bounds(p, O.grid_uniform(ndim, N), start, n)
    g = math.exp(float(a @ y[j0]))
    # (no other point within the band, 2^-20, of either cut)
    assert np.sum(np.abs(y[:, 0] - u[0]) <= 2.0 ** -20) == 1
    assert np.all(np.abs(y[:, 1] - u[1]) > 2.0 ** -20)
    assert r.B1[0] == pytest.approx(g, rel=1e-15)
    assert r.B2[0] == pytest.approx(g * g, rel=1e-15)
    # the oracle's own decision is the FP64 one: x = u is inside
    inside = (y[:, 0] <= u[0]) & (y[:, 1] <= u[1])
    assert r.S1[0] == pytest.approx(np.sum(np.exp(y[inside] @ a)), rel=1e-14)
    # a cut on the other axis that puts the point outside anyway removes it
    u2 = u.copy()
    u2[1] = y[j0, 1] - 1e-3
    r2 = O.sample_bounds(_problem(ndim, [O.DISCONTINUOUS], a, u2, nbins=N, bits=23),
                         O.grid_uniform(ndim, N), start, n)
    assert r2.B1[0] == 0.0 and r2.B2[0] == 0.0
    # an FP64 comparison (52-bit coordinates, no band) has no boundary mass
    r3 = O.sample_bounds(_problem(ndim, [O.DISCONTINUOUS], a, u, nbins=N, bits=52),
                         O.grid_uniform(ndim, N), start, n)
    assert r3.B1[0] == 0.0


def test_boundary_band_width_is_sixteen_binary32_units():
    # the band is |x - u| <= 2^-20 (16 units of 2^-24): a cut 0.9 band
    # widths from the point keeps it ambiguous, 1.1 widths does not
    ndim, N, start, n, j0 = 2, 32, 1, 32, 9
    a = np.array([0.5, 0.5])
    y = _scipy_points(ndim, start, n)
    band = 2.0 ** -20
    got = []
    for t in (0.9, 1.1, -0.9, -1.1):
        u = np.array([y[j0, 0] + t * band, 1.0])
        p = _problem(ndim, [O.DISCONTINUOUS], a, u, nbins=N, bits=23)
        got.append(O.sample_bounds(p, O.grid_uniform(ndim, N), start, n).B1[0] > 0)
    assert got == [True, False, True, False]


def test_abs_sum_bounds_the_sum():
    # sum |J f| equals S1 bit for bit for a positive integrand and exceeds
    # |S1| for an oscillatory one; no family but the discontinuous one has
    # boundary mass
    e = _random_grid(4, 32, 3)
    fams = [O.GAUSSIAN, O.OSCILLATORY, O.CORNER_PEAK, O.C0]
    p = _problem(4, fams, [2.0, 3.0, 1.0, 0.5], [0.3, 0.6, 0.5, 0.45], nbins=32, bits=23)
    p.a[1] *= 4
    r = O.sample_bounds(p, e, 1, 20000, nthreads=3)
    assert r.A1[0] == r.S1[0] and r.A1[2] == r.S1[2] and r.A1[3] == r.S1[3]
    assert r.A1[1] > abs(r.S1[1])
    assert np.all(r.B1 == 0) and np.all(r.B2 == 0)
    S1, S2, H = O.sample(p, e, 1, 20000)
    np.testing.assert_allclose(S1, r.S1, rtol=1e-14)
    np.testing.assert_allclose(H, r.H, rtol=1e-14)


def test_boundary_mass_is_small_and_scales_with_the_band():
    # on a random grid the ambiguous points are those within ~1e-6 of a
    # cut: their mass is a small fraction of the pass, and it shrinks with
    # the band (band_bits 53: a band of 2^-49)
    a, u = [0.5, 0.5, 0.5], [0.3, 0.7, 0.5]
    e = _random_grid(3, 64, 2)
    n = 200000
    p = _problem(3, [O.DISCONTINUOUS], a, u, nbins=64, bits=23)
    r = O.sample_bounds(p, e, 1, n, nthreads=4)
    assert 0.0 <= r.B1[0] <= 1e-3 * r.S1[0]
    p.band_bits = 53
    assert O.sample_bounds(p, e, 1, n, nthreads=4).B1[0] <= r.B1[0]


# ---------------------------------------------------------------- refinement
def test_equal_histogram_leaves_grid_unchanged_exactly():
    for nbins in (8, 64, 256):
        e = O.grid_uniform(3, nbins)
        assert np.array_equal(O.refine(e, np.full((3, nbins), 2.5)), e)
    e = _random_grid(2, 50, 9)
    assert np.array_equal(O.refine(e, np.full((2, 50), 0.125)), e)


def test_zero_or_nonfinite_histogram_leaves_grid_unchanged():
    e = _random_grid(2, 16, 4)
    assert np.array_equal(O.refine(e, np.zeros((2, 16))), e)
    H = np.ones((2, 16))
    H[1, 3] = np.nan
    out = O.refine(e, H)
    assert np.array_equal(out[1], e[1])


def test_refine_is_scale_invariant():
    rng = np.random.default_rng(3)
    e = _random_grid(3, 32, 1)
    H = rng.random((3, 32))
    assert np.array_equal(O.refine(e, H), O.refine(e, 4.0 * H))


def test_refine_mirror_symmetry():
    rng = np.random.default_rng(4)
    N = 40
    e = O.grid_uniform(1, N)
    H = rng.random((1, N))
    a = O.refine(e, H)
    b = O.refine(e, H[:, ::-1].copy())
    np.testing.assert_allclose(b[0], 1.0 - a[0][::-1], atol=2e-15)


def test_refine_keeps_monotone_partition_and_concentrates():
    N = 64
    e = O.grid_uniform(2, N)
    x = (np.arange(N) + 0.5) / N
    H = np.vstack([np.exp(-50 * (x - 0.3) ** 2), np.exp(-50 * (x - 0.8) ** 2)])
    out = O.refine(e, H)
    w = np.diff(out, axis=1)
    assert np.all(w > 0) and np.all(out[:, 0] == 0) and np.all(out[:, -1] == 1)
    # narrowest bins sit at the peak of the histogram
    mid = 0.5 * (out[:, 1:] + out[:, :-1])
    assert abs(mid[0, np.argmin(w[0])] - 0.3) < 0.05
    assert abs(mid[1, np.argmin(w[1])] - 0.8) < 0.05


def test_rebin_gives_equal_shares_of_the_weight():
    # the piecewise-linear cumulative weight at new edge m is m R / N.
    rng = np.random.default_rng(8)
    N = 50
    e = _random_grid(2, N, 12)
    r = rng.random((2, N))
    r[0, 10:14] = 0.0
    out = O.rebin(e, r)
    for d in range(2):
        C = np.concatenate([[0.0], np.cumsum(r[d])])
        share = np.interp(out[d], e[d], C)
        np.testing.assert_allclose(share, np.arange(N + 1) * C[-1] / N, rtol=1e-13, atol=1e-13)


def test_refine_worked_three_bin_example():
    # H = (0, 1, 0) on three equal bins.  Smoothing: h = (1/2, 1/3, 1/2),
    # s = 4/3.  Compression (alpha = 3/2): r_0 = r_2 = ((5/8)/ln(8/3))^1.5,
    # r_1 = ((3/4)/ln 4)^1.5.  Rebinning puts new edge 1 where the weight
    # r_0 x (3 x) reaches R/3, inside the first old bin, and edge 2 by
    # mirror symmetry.
    r0 = (0.625 / math.log(8.0 / 3.0)) ** 1.5
    r1 = (0.75 / math.log(4.0)) ** 1.5
    R = 2 * r0 + r1
    x1 = (R / 3.0) / r0 / 3.0
    out = O.refine(O.grid_uniform(1, 3), np.array([[0.0, 1.0, 0.0]]))
    assert out[0, 1] == pytest.approx(x1, rel=1e-14)
    assert out[0, 2] == pytest.approx(1.0 - x1, rel=1e-14)


# ---------------------------------------------------------------- combination
def test_chi2_cdf_against_regularized_gamma():
    for k in range(1, 41):
        for x in (0.01, 0.5, 1.0, 3.0, 10.0, 40.0, 120.0):
            assert O.chi2_cdf(x, k) == pytest.approx(special.gammainc(k / 2, x / 2),
                                                      rel=1e-12, abs=1e-15)
    assert O.chi2_cdf(0.0, 3) == 0.0


def test_combine_worked_examples():
    mean, err, chi2, prob = O.combine([1.0, 3.0], [1.0, 1.0])
    assert (mean, chi2) == (2.0, 2.0)
    assert err == pytest.approx(1 / math.sqrt(2), rel=1e-15)
    assert prob == pytest.approx(math.erf(1.0), rel=1e-14)
    mean, err, chi2, prob = O.combine([1.0, 2.0], [1.0, 4.0])
    assert mean == pytest.approx(1.2, rel=1e-15)
    assert err == pytest.approx(1 / math.sqrt(1.25), rel=1e-15)
    assert chi2 == pytest.approx(0.2, rel=1e-14)
    assert prob == pytest.approx(stats.chi2.cdf(0.2, 1), rel=1e-13)
    assert O.combine([5.0], [2.0]) == (5.0, math.sqrt(2.0), 0.0, 0.0)
    assert O.combine([1.0, 2.0, 4.0], [1.0, 0.0, 1.0]) == (7.0 / 3.0, 0.0, 0.0, 0.0)


# ---------------------------------------------------------------- driver
def test_vegas_gaussian3d_within_three_sigma():
    p = _problem(3, [O.GAUSSIAN], 5.0, 0.5, nbins=50)
    r = O.vegas(p, maxeval=10 * 10 ** 4, nstart=10 ** 4)
    exact = (math.sqrt(math.pi) / 5.0 * math.erf(2.5)) ** 3
    assert r.niter == 10 and r.neval == 10 ** 5 and r.fail == 1
    assert abs(r.integral[0] - exact) < 3 * r.error[0]
    assert 0.0 <= r.prob[0] <= 1.0


def test_vegas_constant_is_exact():
    p = _problem(4, [O.CONST], 1.0, 0.5, nbins=64)
    r = O.vegas(p, epsrel=1e-3, maxeval=10 ** 5, nstart=1000)
    assert r.integral[0] == 1.0 and r.error[0] == 0.0 and r.fail == 0 and r.niter == 1


def test_vegas_sample_schedule_and_maxeval():
    p = _problem(2, [O.GAUSSIAN], 2.0, 0.5, nbins=16)
    r = O.vegas(p, maxeval=5000, nstart=1000, nincrease=500)
    assert r.niter == 3 and r.neval == 1000 + 1500 + 2000 and r.fail == 1


def test_vegas_stops_at_requested_accuracy():
    p = _problem(2, [O.GAUSSIAN], 2.0, 0.5, nbins=32)
    r = O.vegas(p, epsrel=1e-3, maxeval=10 ** 6, nstart=2000, nincrease=1000)
    assert r.fail == 0 and r.error[0] <= 1e-3 * abs(r.integral[0])
    assert r.neval == sum(2000 + 1000 * j for j in range(r.niter))
    # and it had not reached it one iteration earlier
    m = r.niter - 1
    if m > 0:
        _, err_prev, _, _ = O.combine(r.iter_I[:m, 0], r.iter_var[:m, 0])
        assert err_prev > 1e-3 * abs(O.combine(r.iter_I[:m, 0], r.iter_var[:m, 0])[0])


def test_vegas_mineval_forces_more_iterations():
    p = _problem(2, [O.GAUSSIAN], 2.0, 0.5, nbins=32)
    r = O.vegas(p, epsrel=1e-1, mineval=8000, maxeval=10 ** 6, nstart=2000)
    assert r.fail == 0 and r.neval == 8000


@pytest.mark.parametrize("fam", [O.OSCILLATORY, O.PRODUCT_PEAK, O.CORNER_PEAK,
                                 O.GAUSSIAN, O.C0, O.DISCONTINUOUS])
def test_vegas_all_families_within_four_sigma(fam):
    rng = np.random.default_rng(100 + fam)
    ndim = 4
    a = rng.uniform(0.5, 2.0, ndim)
    a *= 4.0 / a.sum()
    u = rng.uniform(0.2, 0.8, ndim)
    p = _problem(ndim, [fam], a, u, nbins=32)
    r = O.vegas(p, maxeval=8 * 4096, nstart=4096)
    exact = p.exact()[0]
    assert abs(r.integral[0] - exact) < 4 * r.error[0] + 1e-12
    assert np.all(np.diff(r.edges, axis=1) > 0)


def test_vegas_multicomponent_drives_grid_by_component0():
    # the grid depends only on component 0: adding components leaves the
    # component-0 result unchanged.
    a, u = [3.0, 2.0, 2.5], [0.5, 0.4, 0.6]
    p1 = _problem(3, [O.GAUSSIAN], a, u, nbins=32)
    p2 = _problem(3, [O.GAUSSIAN, O.OSCILLATORY, O.C0], a, u, nbins=32)
    r1 = O.vegas(p1, maxeval=5 * 3000, nstart=3000)
    r2 = O.vegas(p2, maxeval=5 * 3000, nstart=3000)
    assert r1.integral[0] == r2.integral[0] and np.array_equal(r1.edges, r2.edges)


def test_iteration_variance_is_the_sample_variance_of_the_mean():
    # var_j = (S2/n - I^2)/(n-1) is the unbiased variance of the mean of
    # the n weighted values g_i = J_i f(x_i); rebuild g_i point by point
    # and let numpy compute it.
    ndim, N, n = 3, 8, 37
    p = _problem(ndim, [O.PRODUCT_PEAK], [2.0, 3.0, 1.5], [0.3, 0.5, 0.7], nbins=N)
    r = O.vegas(p, maxeval=n, nstart=n)
    e = O.grid_uniform(ndim, N)
    Y = O.sobol_coords(ndim, 1, n, 52)
    g = []
    for j in range(n):
        x, J, _ = O.map_point(e, Y[:, j], 52)
        g.append(J * O.genz(O.PRODUCT_PEAK, p.a[0], p.u[0], x))
    g = np.array(g)
    assert r.iter_I[0, 0] == pytest.approx(g.mean(), rel=1e-14)
    assert r.iter_var[0, 0] == pytest.approx(np.var(g, ddof=1) / n, rel=1e-12)
