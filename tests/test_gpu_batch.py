"""GPU tests of the batched persistent path (cv_batch_*): every integral of
a batch against the same integral run alone (cv_vegas, FP32 path) and
against the Genz closed forms within 3 sigma; uneven sizes, mixed dimensions and
bin counts, early stops, and the tile autotuner."""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1408_6373_gb300 as cg  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cg.build_library()
    c = cg.Context(0)
    yield c
    c.close()


def _specs(count, seed, nmin=300, nmax=60000, iters=5, nbins_choices=(64, 32, 50)):
    rng = np.random.default_rng(seed)
    specs, probs = [], []
    for i in range(count):
        ndim = int(rng.integers(1, 17))
        fam = int(rng.integers(0, 6))
        a = 0.5 + rng.random(ndim)
        u = rng.random(ndim)
        n = int(np.exp(rng.uniform(np.log(nmin), np.log(nmax))))
        nbins = int(rng.choice(nbins_choices))
        g = cg.genz(ndim, [fam], a, u)
        specs.append(cg.spec(g, nbins=nbins, maxeval=iters * n, nstart=n))
        probs.append(O.Problem(ndim, [fam], a[None], u[None], nbins=nbins, bits=23))
    return specs, probs


def test_batch_matches_single_runs(ctx):
    specs, probs = _specs(24, 1)
    res = ctx.batch_vegas(specs)
    for sp, r, p in zip(specs, res, probs):
        single = ctx.vegas(sp.g, flags=0, maxeval=sp.maxeval, nstart=sp.nstart, nbins=sp.nbins)
        assert (r.neval, r.fail) == (single.neval, single.fail)
        # same points, summed in another order in FP32: the grids drift apart at
        # the 1e-7 level, far below the statistical error
        assert abs(r.integral[0] - single.integral[0]) <= 2e-5 * abs(single.integral[0]) + 1e-2 * single.error[0]
        exact = p.exact()[0]
        assert abs(r.integral[0] - exact) <= 3 * r.error[0] + 2e-6 * abs(exact) + 1e-12


def test_batch_small_power_of_two_bins(ctx):
    # 2..16 bins take the general map (the bit-permuted form starts at 32)
    specs, probs = _specs(12, 11, nbins_choices=(2, 4, 8, 16, 32))
    res = ctx.batch_vegas(specs)
    for sp, r, p in zip(specs, res, probs):
        single = ctx.vegas(sp.g, flags=0, maxeval=sp.maxeval, nstart=sp.nstart, nbins=sp.nbins)
        assert (r.neval, r.fail) == (single.neval, single.fail)
        assert abs(r.integral[0] - single.integral[0]) <= 2e-5 * abs(single.integral[0]) + 1e-2 * single.error[0]
        exact = p.exact()[0]
        assert abs(r.integral[0] - exact) <= 3 * r.error[0] + 2e-6 * abs(exact) + 1e-12


def _bits(r):
    return [np.float64(v).view(np.uint64) for v in (r.integral[0], r.error[0], r.prob[0])]


def _private_hist(sp):
    # power-of-two bins from 32 on: warp-private histogram copies, plain
    # updates in a fixed order (other bin counts add into a warp's copy
    # with shared-memory atomics, in hardware order)
    return sp.nbins >= 32 and sp.nbins & (sp.nbins - 1) == 0


def test_batch_alone_equals_in_mix(ctx):
    # an integral's tiles and their sums do not depend on the rest of the
    # batch, and its tiles' partial rows are added in tile order: alone and
    # in the mix give the same bits
    specs, _ = _specs(10, 2)
    mix = ctx.batch_vegas(specs)
    checked = 0
    for k in range(len(specs)):
        alone = ctx.batch_vegas([specs[k]])[0]
        assert (alone.neval, alone.fail, alone.iterations) == (mix[k].neval, mix[k].fail, mix[k].iterations)
        if _private_hist(specs[k]):
            assert _bits(alone) == _bits(mix[k]), k
            checked += 1
        else:
            assert alone.integral[0] == pytest.approx(mix[k].integral[0], rel=1e-10, abs=1e-15)
            assert alone.error[0] == pytest.approx(mix[k].error[0], rel=1e-8)
    assert checked >= 3


def test_batch_accuracy_goals_stop_each_integral(ctx):
    specs, _ = _specs(12, 3, nmin=2000, nmax=20000, iters=30)
    for i, sp in enumerate(specs):
        if i % 2 == 0:
            sp.epsrel = 1e-3
            sp.nincrease = 1000
            sp.maxeval = 10 ** 6
    res = ctx.batch_vegas(specs)
    for i, (sp, r) in enumerate(zip(specs, res)):
        alone = ctx.batch_vegas([sp])[0]
        assert (r.neval, r.fail, r.iterations) == (alone.neval, alone.fail, alone.iterations)
        if i % 2 == 0 and r.fail == 0:
            assert r.error[0] <= 1e-3 * abs(r.integral[0])
        if i % 2 == 1:
            assert r.iterations == 30 and r.fail == 1


def test_batch_rerun_and_autotune_keep_results(ctx):
    specs, _ = _specs(16, 4, nmin=1000, nmax=100000, iters=4)
    B = ctx.batch(specs)
    B.run()
    r1 = B.results()
    # the same run again: the same bits (no floating-point atomics)
    B.run()
    r0 = B.results()
    for sp, a, b in zip(specs, r1, r0):
        if _private_hist(sp):
            assert _bits(a) == _bits(b)
    B.autotune()
    assert 2048 <= B.tile_points(10 ** 6) <= 4096 * 32
    B.run()
    r2 = B.results()
    for a, b in zip(r1, r2):
        assert a.neval == b.neval
        assert a.integral[0] == pytest.approx(b.integral[0], rel=2e-5)
    assert B.kernels_per_run() > 0
    B.close()


def test_batch_tiny_and_ragged_sizes(ctx):
    g = cg.genz(3, [cg.CONST], 1.0, 0.5)
    specs = [cg.spec(g, nbins=32, maxeval=2 * n, nstart=n) for n in (2, 31, 33, 1000)]
    for r, sp in zip(ctx.batch_vegas(specs), specs):
        assert r.integral[0] == 1.0 and r.error[0] == 0.0 and r.neval == sp.nstart
