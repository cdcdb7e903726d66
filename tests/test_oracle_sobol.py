"""Pins for the oracle's Sobol generator (Sobol 1967; Gray-code order of
Antonov & Saleev 1979; direction numbers by the Bratley-Fox 1988
recurrence on the Joe-Kuo primitive polynomials).

The oracle is checked against things other than itself: scipy's
unscrambled Sobol points (a library special case), the digital-net
property every Sobol sequence has, and the closed form of dimension 0
(van der Corput in Gray-code order)."""
import numpy as np
import pytest
from scipy.stats import qmc

import oracle as O


@pytest.mark.parametrize("ndim", [1, 2, 8, 32, 40])
def test_equals_scipy_unscrambled_first_points(ndim):
    # scipy with bits=52 keeps the top 52 bits of each direction word, so
    # its points are our words shifted right by 12 (b = 52), exactly.
    n = 2048
    Y = O.sobol_coords(ndim, 0, n, 52)
    ref = qmc.Sobol(ndim, scramble=False, bits=52).random(n) * 2.0 ** 52
    assert np.array_equal(Y.T.astype(np.float64), ref)


@pytest.mark.parametrize("start", [2 ** 20 - 7, 3 * 2 ** 22 + 11])
def test_equals_scipy_after_fast_forward(start):
    # (scipy's fast_forward needs its 32-bit engine; compare the top 32 bits)
    ndim, n = 12, 64
    Y = O.sobol_coords(ndim, start, n, 32)
    eng = qmc.Sobol(ndim, scramble=False, bits=32)
    eng.fast_forward(start)
    ref = eng.random(n) * 2.0 ** 32
    assert np.array_equal(Y.T.astype(np.float64), ref)


def test_fp32_path_bits_are_the_top_bits():
    # b = 23 (FP32 path) takes the top 23 bits of the same words.
    Y52 = O.sobol_coords(6, 1, 5000, 52)
    Y23 = O.sobol_coords(6, 1, 5000, 23)
    assert np.array_equal(Y52 >> np.uint64(29), Y23)


def _bitreverse64(x: int) -> int:
    return int(format(x, "064b")[::-1], 2)


def test_dimension0_is_van_der_corput_in_gray_order():
    idx = list(range(0, 300)) + [2 ** 40 + 17, 2 ** 62 + 5]
    X = O.sobol_words(1, idx)
    for j, i in enumerate(idx):
        g = i ^ (i >> 1)
        assert int(X[0, j]) == _bitreverse64(g)


@pytest.mark.parametrize("m", [1, 4, 7, 10])
def test_one_dimensional_projections_are_0_m_1_nets(m):
    # Every aligned block of 2^m points has exactly one point in each
    # interval [j/2^m, (j+1)/2^m) in every coordinate.
    ndim, nblocks = 16, 3
    Y = O.sobol_coords(ndim, 0, nblocks * 2 ** m, 52)
    cells = (Y >> np.uint64(52 - m)).astype(np.int64)
    for b in range(nblocks):
        blk = cells[:, b * 2 ** m:(b + 1) * 2 ** m]
        for d in range(ndim):
            assert np.array_equal(np.sort(blk[d]), np.arange(2 ** m))


@pytest.mark.parametrize("m", [2, 6, 9, 12])
def test_first_two_dimensions_form_0_m_2_nets(m):
    # Dimensions 0 and 1 of the Sobol sequence are a (0,2)-sequence: every
    # aligned block of 2^m points puts one point in each elementary box of
    # area 2^-m, 2^-a x 2^-(m-a), for every a in 0..m.
    Y = O.sobol_coords(2, 3 * 2 ** m, 2 ** m, 52)
    for a in range(m + 1):
        cx = (Y[0] >> np.uint64(52 - a)).astype(np.int64) if a else np.zeros(2 ** m, np.int64)
        cy = (Y[1] >> np.uint64(52 - (m - a))).astype(np.int64) if m - a else np.zeros(2 ** m, np.int64)
        boxes = cx * 2 ** (m - a) + cy
        assert np.array_equal(np.sort(boxes), np.arange(2 ** m))


def test_gray_order_blocks_match_natural_order_sets():
    # An aligned block of Gray-code indices holds the same point set as the
    # aligned natural-order block it maps onto; this is what lets a warp of
    # 32 aligned indices see 32 distinct 1/32-strata.
    V = O.sobol_directions(4)
    q, m = 37, 5
    idx = np.arange(q * 2 ** m, (q + 1) * 2 ** m, dtype=np.uint64)
    gray_pts = O.sobol_words(4, idx, V)
    g = idx ^ (idx >> np.uint64(1))
    # natural-order point with index n has word XOR of V over bits of n
    nat = np.zeros_like(gray_pts)
    for j, gi in enumerate(g):
        for d in range(4):
            acc = np.uint64(0)
            for k in range(64):
                if (int(gi) >> k) & 1:
                    acc ^= V[d, k]
            nat[d, j] = acc
    assert np.array_equal(np.sort(gray_pts, axis=1), np.sort(nat, axis=1))


def test_direction_words_are_odd_fractions():
    # V[d,k] = m_{k+1}/2^{k+1} with m odd and < 2^{k+1}: the lowest set bit
    # of V[d,k] is bit 63-k.
    V = O.sobol_directions(32)
    for k in range(64):
        low = V[:, k] & (~V[:, k] + np.uint64(1))
        assert np.all(low == np.uint64(1) << np.uint64(63 - k))


def test_rejects_bad_initial_numbers():
    poly, vinit = O.joe_kuo_table()
    bad = vinit.copy()
    bad[3, 0] = 2  # even initial number
    with pytest.raises(ValueError):
        O.sobol_directions(4, poly, bad)
