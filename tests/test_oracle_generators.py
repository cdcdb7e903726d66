"""Pins of the oracle's counter-based generator and its point generators.

- Philox4x64-10 (Salmon et al., SC 2011) against numpy's independent
  implementation (numpy's generator emits the block of counter + 1).
- Pseudo-random points are Philox words (i, d/4, 0, 0)[d mod 4].
- Scrambled Sobol points are scipy's unscrambled Sobol points XOR a
  per-dimension digital shift, Philox word (0, d/4, 1, 0)[d mod 4]; the
  shift keeps the (0, m, 1)-net property of every coordinate.
- Pseudo-random coordinates are uniform and uncorrelated; scrambled
  replicates give an unbiased estimate with far smaller variance than
  pseudo-random sampling (randomized QMC).
"""
import math

import numpy as np
import pytest

import oracle as O

M64 = (1 << 64) - 1


def numpy_philox(ctr, key):
    """numpy's Philox4x64-10 block of counter ctr (numpy advances its
    counter by one before each block, so it is seeded with ctr - 1)."""
    c = list(ctr)
    for j in range(4):  # c - 1 with borrow
        if c[j] > 0:
            c[j] -= 1
            break
        c[j] = M64
    bg = np.random.Philox(counter=np.array(c, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    return [int(v) for v in bg.random_raw(4)]


def test_philox_matches_numpy():
    rng = np.random.default_rng(5)
    cases = [([1, 0, 0, 0], [0, 0]), ([0, 1, 0, 0], [3, 4]), ([0, 0, 1, 0], [M64, M64]),
             ([M64, M64, M64, M64], [1, 2])]
    for _ in range(40):
        cases.append((list(map(int, rng.integers(0, 2 ** 63, 4))), list(map(int, rng.integers(0, 2 ** 63, 2)))))
    for ctr, key in cases:
        assert [int(v) for v in O.philox(ctr, key)] == numpy_philox(ctr, key), (ctr, key)


@pytest.mark.parametrize("seed", [0, 1, 987654321])
def test_pseudo_words_are_philox_words(seed):
    ndim = 7
    idx = [1, 2, 3, 1000, 2 ** 33 + 5]
    W = O.point_words(O.PSEUDO, seed, ndim, idx)
    for j, i in enumerate(idx):
        for d in range(ndim):
            assert int(W[d, j]) == numpy_philox([i, d // 4, 0, 0], [seed, 0])[d % 4]


@pytest.mark.parametrize("seed", [1, 42])
def test_scrambled_is_scipy_sobol_xor_shift(seed):
    qmc = pytest.importorskip("scipy.stats.qmc")
    ndim, n = 9, 512
    ref = qmc.Sobol(ndim, scramble=False, bits=52).random_base2(10)[: n + 1]  # indices 0..n
    W = O.point_words(O.SCRAMBLED, seed, ndim, range(1, n + 1))
    for d in range(ndim):
        shift = numpy_philox([0, d // 4, 1, 0], [seed, 0])[d % 4]
        for j in range(n):
            sobol = int(round(ref[j + 1, d] * 2.0 ** 52)) << 12
            assert int(W[d, j]) == sobol ^ shift


def test_digital_shift_keeps_the_net_property():
    # every aligned block of 2^m points has one point in each 1/2^m interval
    ndim, bits = 5, 52
    for m in (4, 8, 11):
        Y = O.point_coords(O.SCRAMBLED, 77, ndim, 3 * 2 ** m, 2 ** m, bits)
        for d in range(ndim):
            strata = (Y[d] >> np.uint64(bits - m)).astype(np.int64)
            assert np.array_equal(np.sort(strata), np.arange(2 ** m))


def test_seeds_change_and_reproduce_points():
    a = O.point_coords(O.SCRAMBLED, 1, 4, 1, 64, 52)
    b = O.point_coords(O.SCRAMBLED, 2, 4, 1, 64, 52)
    assert not np.array_equal(a, b)
    assert np.array_equal(a, O.point_coords(O.SCRAMBLED, 1, 4, 1, 64, 52))
    assert not np.array_equal(O.point_coords(O.PSEUDO, 1, 4, 1, 64, 52),
                              O.point_coords(O.PSEUDO, 2, 4, 1, 64, 52))


def test_pseudo_coordinates_uniform_and_uncorrelated():
    ndim, n, nb = 6, 1 << 16, 64
    Y = O.point_coords(O.PSEUDO, 2024, ndim, 1, n, 52).astype(np.float64) * 2.0 ** -52
    for d in range(ndim):
        counts = np.bincount((Y[d] * nb).astype(int), minlength=nb)
        chi2 = ((counts - n / nb) ** 2 / (n / nb)).sum()
        assert chi2 < nb + 8 * math.sqrt(2 * nb), (d, chi2)
        assert abs(Y[d].mean() - 0.5) < 6 * math.sqrt(1 / 12 / n)
    C = np.corrcoef(Y)
    assert np.max(np.abs(C - np.eye(ndim))) < 6 / math.sqrt(n)


def _gauss_problem(gen, seed):
    a, u = np.array([[3.0, 2.0, 4.0]]), np.array([[0.4, 0.6, 0.5]])
    return O.Problem(3, [O.GAUSSIAN], a, u, nbins=16, bits=52, gen=gen, seed=seed)


def test_randomized_qmc_replicates():
    # one pass on the uniform grid: scrambled replicates are unbiased and
    # their spread is far below that of pseudo-random replicates
    n, R = 4096, 24
    edges = O.grid_uniform(3, 16)
    exact = _gauss_problem(O.SOBOL, 0).exact()[0]
    est = {}
    for gen in (O.SCRAMBLED, O.PSEUDO):
        est[gen] = np.array([O.sample(_gauss_problem(gen, s + 1), edges, 1, n)[0][0] / n for s in range(R)])
    m, sd = est[O.SCRAMBLED].mean(), est[O.SCRAMBLED].std(ddof=1)
    assert abs(m - exact) < 5 * sd / math.sqrt(R)
    assert sd < 0.2 * est[O.PSEUDO].std(ddof=1)
    assert abs(est[O.PSEUDO].mean() - exact) < 5 * est[O.PSEUDO].std(ddof=1) / math.sqrt(R)


@pytest.mark.parametrize("gen", [O.SCRAMBLED, O.PSEUDO])
def test_vegas_with_random_points_meets_the_closed_form(gen):
    p = _gauss_problem(gen, 11)
    r = O.vegas(p, maxeval=8 * 20000, nstart=20000)
    assert abs(r.integral[0] - p.exact()[0]) < 4 * r.error[0]


def test_delay_leaves_values_unchanged():
    # the integrand-cost knob adds work, never value
    edges = O.grid_uniform(3, 16)
    base = O.sample(_gauss_problem(O.SOBOL, 0), edges, 1, 5000)
    p = _gauss_problem(O.SOBOL, 0)
    p.delay = 100
    slow = O.sample(p, edges, 1, 5000)
    for x, y in zip(base, slow):
        assert np.array_equal(x, y)
