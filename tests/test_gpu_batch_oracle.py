"""The batched persistent sampling kernel (cv_batch_*, the kernel behind the
4096-integral batch and the serving loop) against the FP64 oracle, element
by element: every integral's first two iterations, read from the batch's
per-iteration log, against the oracle's sampling pass on the same grid --
the uniform grid for the first, the grid the batch's own first refinement
produced for the second.

72 integrals cover 2..32 dimensions (both sides of the 16/17 kernel
boundary), all six Genz families, 50, 64, 128 and 256 bins (256 up to 22
dimensions, the batched path's shared-memory limit), and iterations of up
to a million points, so that tiles reach the largest size; 24 more have
2..4 components of mixed families (the served requests' form) and half of
them digitally shifted Sobol points.  The FP32
tolerances are those of tests/tolerances.py (1e-6 of sum |J f| plus the
boundary mass for I, the implied variance bound)."""
import os

import numpy as np
import pytest

import oracle as O
from tests.tolerances import check_fp32_iteration

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1408_6373_gb300 as cg  # noqa: E402
from paper_1408_6373_gb300 import workloads as W  # noqa: E402

THREADS = os.cpu_count() or 1
COUNT = 72


def _items():
    rng = np.random.default_rng(2025)
    out = []
    for i in range(COUNT):
        ndim = 2 + (5 * i) % 31
        fam = i % 6
        nbins = (64, 50, 256)[i % 3]
        if nbins == 256 and ndim > 22:
            nbins = 128
        n = 10 ** 6 if i % 9 == 0 else int(np.exp(rng.uniform(np.log(2000), np.log(300000))))
        a = 0.5 + rng.random(ndim)
        u = rng.random(ndim)
        if fam == O.CORNER_PEAK:
            a = W.fp32_corner_peak(a)
        out.append((ndim, fam, nbins, n, a, u))
    return out


def _specs(items, iters):
    return [cg.spec(cg.genz(nd, [f], a, u), nbins=N, maxeval=iters * n, nstart=n)
            for nd, f, N, n, a, u in items]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cg.build_library()
    c = cg.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def runs(ctx):
    items = _items()
    B2 = ctx.batch(_specs(items, 2))
    B2.run()
    logs = [B2.log(i, 2) for i in range(COUNT)]
    assert B2.tile_points(10 ** 6) >= 32768  # the million-point iterations use full tiles
    B2.close()
    B1 = ctx.batch(_specs(items, 1))
    B1.run()
    grids = [B1.grid(i) for i in range(COUNT)]
    B1.close()
    return items, logs, grids


def _oracle(item, edges, start):
    nd, f, N, n, a, u = item
    p = O.Problem(nd, [f], a[None], u[None], nbins=N, bits=23)
    return O.sample_bounds(p, edges, start, n, nthreads=THREADS)


def test_batched_first_iteration_matches_oracle(runs):
    items, logs, _ = runs
    for i, item in enumerate(items):
        nd, f, N, n, _, _ = item
        (lI, lV) = logs[i]
        ob = _oracle(item, O.grid_uniform(nd, N), 1)
        check_fp32_iteration(lI[0], lV[0], ob, n, what=(i, nd, f, N, n))


def test_batched_second_iteration_on_refined_grid_matches_oracle(runs):
    items, logs, grids = runs
    for i, item in enumerate(items):
        nd, f, N, n, _, _ = item
        (lI, lV) = logs[i]
        assert np.all(np.diff(grids[i], axis=1) > 0)
        ob = _oracle(item, grids[i], 1 + n)
        check_fp32_iteration(lI[1], lV[1], ob, n, what=(i, nd, f, N, n))


def test_batched_refinement_follows_the_oracle(runs):
    # the batch's refined grid against the oracle's refinement of the
    # oracle's own histogram: they differ only through the FP32 histogram
    # (1e-5 of a bin's share at most), so edges agree to 1e-5 of the bin.
    # A pass with boundary mass (a point a binary32 evaluation may put on
    # the other side of a cut) can move a whole point's weight between
    # bins, so those are left to the sum checks above.
    items, _, grids = runs
    checked = 0
    for i, item in enumerate(items):
        nd, f, N, n, _, _ = item
        if n < 50000:
            continue
        ob = _oracle(item, O.grid_uniform(nd, N), 1)
        if ob.B2[0] > 0:
            continue
        ref = O.refine(O.grid_uniform(nd, N), ob.H)
        assert np.max(np.abs(grids[i] - ref)) <= 1e-5 / N, (i, nd, f, N)
        checked += 1
    assert checked >= 10


def test_autotuned_tiles_and_alone_runs_match_oracle(ctx, runs):
    # other tile sizes group the FP32 sums differently; an integral run alone
    # has the same tiles as in the mix
    items, logs, _ = runs
    B = ctx.batch(_specs(items, 2))
    B.autotune()
    B.run()
    for i in range(0, COUNT, 4):
        lI, lV = B.log(i, 2)
        nd, f, N, n, _, _ = items[i]
        ob = _oracle(items[i], O.grid_uniform(nd, N), 1)
        check_fp32_iteration(lI[0], lV[0], ob, n, what=("autotuned", i))
    B.close()
    for i in (0, 17, 45):
        A = ctx.batch(_specs([items[i]], 2))
        A.run()
        aI, aV = A.log(0, 2)
        A.close()
        # (power-of-two bins: warp-private histograms, and the tiles' partial
        # rows added in tile order: the same bits)
        np.testing.assert_array_equal(aI, logs[i][0])
        np.testing.assert_array_equal(aV, logs[i][1])


# Multi-component integrals (the general policy of the batched kernel, as
# the server runs them) and digitally shifted Sobol points, against the
# oracle's first pass on the uniform grid: 2..4 components of mixed
# families, 2..32 dimensions, 50, 64 and 128 bins.
def _multi_items():
    rng = np.random.default_rng(77)
    out = []
    for i in range(24):
        ndim = 2 + (7 * i) % 31
        ncomp = 2 + i % 3
        fams = [int(f) for f in rng.integers(0, 6, ncomp)]
        nbins = (64, 50, 128)[i % 3]
        n = int(np.exp(rng.uniform(np.log(5000), np.log(200000))))
        a = 0.5 + rng.random((ncomp, ndim))
        u = rng.random((ncomp, ndim))
        for c in range(ncomp):
            if fams[c] == O.CORNER_PEAK:
                a[c] = W.fp32_corner_peak(a[c])
        seed = 0 if i % 2 == 0 else 100 + i
        out.append((ndim, fams, nbins, n, a, u, seed))
    return out


def test_batched_multicomponent_and_scrambled_first_iteration_match_oracle(ctx):
    items = _multi_items()
    specs = [cg.spec(cg.genz(nd, fams, a, u), nbins=N, maxeval=n, nstart=n,
                     flags=cg.SCRAMBLE if seed else 0, seed=seed)
             for nd, fams, N, n, a, u, seed in items]
    B = ctx.batch(specs)
    B.run()
    logs = [B.log(i, 1) for i in range(len(items))]
    B.close()
    for i, (nd, fams, N, n, a, u, seed) in enumerate(items):
        p = O.Problem(nd, fams, a, u, nbins=N, bits=23, gen=O.SCRAMBLED if seed else O.SOBOL, seed=seed)
        ob = O.sample_bounds(p, O.grid_uniform(nd, N), 1, n, nthreads=THREADS)
        lI, lV = logs[i]
        check_fp32_iteration(lI[0], lV[0], ob, n, what=(i, nd, fams, N, n, seed))
