"""GPU parity of the scrambled (randomized QMC) and pseudo-random point
generators against the oracle, through the C ABI.

Tolerances as in the Sobol parity tests: coordinates bit-exact; FP64 sums
within 1e-12; FP32 sums within 1e-6 of sqrt(n S2), the histogram within
1e-5 of its row maximum (the oracle decides float branches in binary32).
"""
import math

import numpy as np
import pytest

import oracle as O
from tests.tolerances import check_fp32_pass

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1408_6373_gb300 as cg  # noqa: E402

GENS = [(cg.SCRAMBLE, O.SCRAMBLED), (cg.PSEUDO, O.PSEUDO)]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cg.build_library()
    c = cg.Context(0)
    yield c
    c.close()


def _random_grid(ndim, nbins, seed):
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.2, 1.0, (ndim, nbins))
    c = np.concatenate([np.zeros((ndim, 1)), np.cumsum(w, axis=1)], axis=1)
    e = c / c[:, -1:]
    e[:, 0], e[:, -1] = 0.0, 1.0
    return e


def _params(ndim, ncomp, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.3, 1.5, (ncomp, ndim))
    a *= min(ndim, 8) / a.sum(axis=1, keepdims=True)
    u = rng.uniform(0.1, 0.9, (ncomp, ndim))
    return a, u


def _gpu_sample(ctx, g, edges, start, n, flags, seed):
    ndim, nbins = edges.shape[0], edges.shape[1] - 1
    e = torch.tensor(edges, dtype=torch.float64, device="cuda")
    S1 = torch.zeros(g.ncomp, dtype=torch.float64, device="cuda")
    S2 = torch.zeros_like(S1)
    H = torch.zeros((ndim, nbins), dtype=torch.float64, device="cuda")
    ctx.sample(g, nbins, e, start, n, flags, S1, S2, H, seed=seed)
    ctx.synchronize()
    return S1.cpu().numpy(), S2.cpu().numpy(), H.cpu().numpy()


@pytest.mark.parametrize("flag,gen", [(0, O.SOBOL)] + GENS)
@pytest.mark.parametrize("bits", [23, 52])
@pytest.mark.parametrize("ndim,start,n", [(7, 1, 3001), (13, 2 ** 33 + 5, 1027), (32, 999, 64)])
def test_points_bit_exact(ctx, flag, gen, bits, ndim, start, n):
    seed = 123456789
    Y = torch.empty((ndim, n), dtype=torch.int64, device="cuda")
    ctx.points(ndim, start, n, bits, flag, seed, Y)
    ctx.synchronize()
    assert np.array_equal(Y.cpu().numpy().view(np.uint64), O.point_coords(gen, seed, ndim, start, n, bits))


@pytest.mark.parametrize("flag,gen", GENS)
def test_sample_fp64_matches_oracle(ctx, flag, gen):
    ndim, N, n, seed = 5, 64, 40000, 31
    a, u = _params(ndim, 2, 5)
    fams = [O.GAUSSIAN, O.OSCILLATORY]
    g = cg.genz(ndim, fams, a, u)
    edges = _random_grid(ndim, N, 7)
    S1, S2, H = _gpu_sample(ctx, g, edges, 17, n, cg.FP64 | flag, seed)
    p = O.Problem(ndim, fams, a, u, nbins=N, bits=52, gen=gen, seed=seed)
    oS1, oS2, oH = O.sample(p, edges, 17, n, nthreads=8)
    np.testing.assert_allclose(S1, oS1, rtol=1e-12, atol=1e-12 * math.sqrt(n * oS2.max()))
    np.testing.assert_allclose(S2, oS2, rtol=1e-12)
    assert np.max(np.abs(H - oH)) <= 1e-12 * oH.max()


@pytest.mark.parametrize("flag,gen", GENS)
@pytest.mark.parametrize("jit", [0, cg.JIT])
@pytest.mark.parametrize("N", [128, 50])
def test_sample_fp32_matches_oracle(ctx, flag, gen, jit, N):
    # N = 128 takes the bit-permuted word layout (the shift is permuted too)
    ndim, n, seed = 8, 200000, 77
    a, u = _params(ndim, 4, 9)
    fams = [O.OSCILLATORY, O.PRODUCT_PEAK, O.DISCONTINUOUS, O.GAUSSIAN]
    g = cg.genz(ndim, fams, a, u)
    edges = _random_grid(ndim, N, 3)
    S1, S2, H = _gpu_sample(ctx, g, edges, 1, n, flag | jit, seed)
    p = O.Problem(ndim, fams, a, u, nbins=N, bits=23, gen=gen, seed=seed)
    check_fp32_pass(S1, S2, H, O.sample_bounds(p, edges, 1, n, nthreads=8), n)


@pytest.mark.parametrize("flag,gen", GENS)
def test_vegas_fp64_matches_oracle(ctx, flag, gen):
    ndim, seed = 4, 2024
    a, u = _params(ndim, 1, 12)
    g = cg.genz(ndim, [O.GAUSSIAN], a, u)
    r = ctx.vegas(g, flags=cg.FP64 | flag, seed=seed, maxeval=6 * 8000, nstart=8000, nbins=64)
    p = O.Problem(ndim, [O.GAUSSIAN], a, u, nbins=64, gen=gen, seed=seed)
    o = O.vegas(p, maxeval=6 * 8000, nstart=8000)
    assert (r.neval, r.fail) == (o.neval, o.fail)
    np.testing.assert_allclose(r.integral[0], o.integral[0], rtol=1e-12)
    np.testing.assert_allclose(r.error[0], o.error[0], rtol=1e-9)


def test_seed_changes_scrambled_results_and_sobol_ignores_it(ctx):
    a, u = _params(3, 1, 4)
    g = cg.genz(3, [O.GAUSSIAN], a, u)
    # (the plain Sobol points do not depend on the seed: equal sums)
    kw = dict(flags=cg.FP64, maxeval=4 * 4000, nstart=4000, nbins=32)
    a1, a2 = ctx.vegas(g, seed=1, **kw).integral[0], ctx.vegas(g, seed=2, **kw).integral[0]
    assert abs(a1 - a2) <= 1e-14 * abs(a1)
    kw["flags"] = cg.FP64 | cg.SCRAMBLE
    b1, b2 = ctx.vegas(g, seed=1, **kw).integral[0], ctx.vegas(g, seed=2, **kw).integral[0]
    assert abs(b1 - b2) > 1e-10 * abs(b1)


def test_randomized_qmc_replicates(ctx):
    # independent scrambles: the replicate mean meets the closed form within
    # its own standard error, and the spread matches Vegas's error estimate
    ndim, R = 6, 16
    a, u = _params(ndim, 1, 21)
    g = cg.genz(ndim, [O.GAUSSIAN], a, u)
    exact = O.genz_exact(O.GAUSSIAN, a[0], u[0])
    est = np.array([ctx.vegas(g, flags=cg.SCRAMBLE, seed=s + 1, maxeval=5 * 200000, nstart=200000,
                              nbins=64).integral[0] for s in range(R)])
    sd = est.std(ddof=1)
    assert abs(est.mean() - exact) < 5 * sd / math.sqrt(R) + 1e-6 * exact
    pseudo = ctx.vegas(g, flags=cg.PSEUDO, seed=5, maxeval=5 * 200000, nstart=200000, nbins=64)
    assert abs(pseudo.integral[0] - exact) < 5 * pseudo.error[0]
    assert sd < pseudo.error[0]  # the quasi-random replicates spread less


def test_scrambled_batch_matches_single_runs(ctx):
    specs = []
    for k in range(6):
        a, u = _params(3 + k, 1, 40 + k)
        specs.append(cg.spec(cg.genz(3 + k, [O.GAUSSIAN], a, u), nbins=64, flags=cg.SCRAMBLE,
                             maxeval=5 * 20000, nstart=20000, seed=100 + k))
    res = ctx.batch_vegas(specs)
    for r, sp in zip(res, specs):
        one = ctx.vegas(sp.g, flags=cg.SCRAMBLE, seed=sp.seed, maxeval=sp.maxeval, nstart=sp.nstart,
                        nbins=sp.nbins)
        assert r.iterations == 5
        assert abs(r.integral[0] - one.integral[0]) <= 1e-4 * abs(one.integral[0]) + 0.1 * one.error[0]


def test_pseudo_refused_where_unsupported(ctx):
    g = cg.genz(3, [O.GAUSSIAN], 1.0, 0.5)
    sp = cg.spec(g, nbins=32, flags=cg.PSEUDO, maxeval=20000, nstart=10000)
    with pytest.raises(cg.CubaGpuError):
        ctx.batch_vegas([sp])
    with pytest.raises(cg.CubaGpuError):
        ctx.vegas(g, flags=cg.SCRAMBLE | cg.PSEUDO, maxeval=20000, nstart=10000, nbins=32)


@pytest.mark.parametrize("flags", [0, cg.JIT, cg.FP64])
def test_delay_leaves_values_unchanged(ctx, flags):
    # the integrand-cost knob (extra multiply-adds per evaluation) changes
    # the cost only (the tolerance leaves room for the order of additions)
    ndim, N, n = 6, 64, 100000
    a, u = _params(ndim, 2, 3)
    edges = _random_grid(ndim, N, 1)
    base = _gpu_sample(ctx, cg.genz(ndim, [O.GAUSSIAN, O.OSCILLATORY], a, u), edges, 1, n, flags, 0)
    slow = _gpu_sample(ctx, cg.genz(ndim, [O.GAUSSIAN, O.OSCILLATORY], a, u, delay=256), edges, 1, n, flags, 0)
    for x, y in zip(base, slow):
        np.testing.assert_allclose(y, x, rtol=1e-13, atol=1e-300)
