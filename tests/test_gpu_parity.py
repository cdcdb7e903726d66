"""GPU parity: the CUDA path (called through the C ABI) against the FP64
oracle, element by element, on the same seeded inputs.

Tolerances:
  - Sobol coordinates and bin assignment: bit-exact (integer arithmetic on
    both sides).
  - FP64 path: S1, S2 within 1e-12 relative (both sides sum 1e4-1e5 terms
    in FP64, the GPU in another order: differences ~1e-15); histogram within
    1e-12 of the row maximum; refined edges within 1e-14 absolute (the GPU's
    refinement uses reciprocal multiplications and CUDA's log, each within
    1.5 ulp, on edges of magnitude <= 1).
  - FP32 path (binary32 point, map and integrand, Kahan sums, FP64
    reduction): S1 within 1e-6 sum |J f| plus the boundary mass of the
    discontinuity band, S2 within 1e-6 S2 plus its boundary mass, the
    iteration variance within the bound those two imply, the histogram
    within 1e-5 of its row maximum (tests/tolerances.py states each bound).
    The oracle decides every branch on its FP64 point.
"""
import math

import numpy as np
import pytest

import oracle as O
from tests.tolerances import check_fp32_pass, check_fp32_iteration

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


def _gpu_sample(ctx, g, edges, start, n, flags):
    ndim, nbins = edges.shape[0], edges.shape[1] - 1
    e = torch.tensor(edges, dtype=torch.float64, device="cuda")
    S1 = torch.zeros(g.ncomp, dtype=torch.float64, device="cuda")
    S2 = torch.zeros_like(S1)
    H = torch.zeros((ndim, nbins), dtype=torch.float64, device="cuda")
    ctx.sample(g, nbins, e, start, n, flags, S1, S2, H)
    ctx.synchronize()
    return S1.cpu().numpy(), S2.cpu().numpy(), H.cpu().numpy()


# ------------------------------------------------------------------ Sobol
@pytest.mark.parametrize("bits", [23, 52])
@pytest.mark.parametrize("ndim,start,n", [
    (1, 0, 1), (3, 1, 10000), (8, 7, 33333), (17, 2 ** 20 + 3, 5000),
    (32, 12345, 70001), (5, 2 ** 40 + 11, 2049), (2, 2 ** 52 - 1000, 1000)])
def test_sobol_bit_exact(ctx, bits, ndim, start, n):
    Y = torch.empty((ndim, n), dtype=torch.int64, device="cuda")
    ctx.sobol(ndim, start, n, bits, Y)
    ctx.synchronize()
    ref = O.sobol_coords(ndim, start, n, bits)
    assert np.array_equal(Y.cpu().numpy().view(np.uint64), ref)


# ------------------------------------------------------------------ FP64 pass
FAMS = [O.OSCILLATORY, O.PRODUCT_PEAK, O.CORNER_PEAK, O.GAUSSIAN, O.C0, O.DISCONTINUOUS, O.CONST]


@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("ndim,nbins,start,n", [(3, 50, 1, 20001), (8, 128, 1000003, 30000)])
def test_sample_fp64_matches_oracle(ctx, fam, ndim, nbins, start, n):
    a, u = _params(ndim, 1, 10 + fam)
    edges = _random_grid(ndim, nbins, fam)
    g = cg.genz(ndim, [fam], a, u)
    S1, S2, H = _gpu_sample(ctx, g, edges, start, n, cg.FP64)
    p = O.Problem(ndim, [fam], a, u, nbins=nbins, bits=52)
    oS1, oS2, oH = O.sample(p, edges, start, n)
    np.testing.assert_allclose(S1, oS1, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(S2, oS2, rtol=1e-12, atol=1e-300)
    scale = np.maximum(oH.max(axis=1, keepdims=True), 1e-300)
    assert np.all(np.abs(H - oH) <= 1e-12 * scale)
    # bins bit-exact: the points that reached each bin are the same
    assert np.array_equal(H == 0, oH == 0)


@pytest.mark.parametrize("ndim,ncomp,nbins", [(1, 2, 2), (4, 4, 64), (13, 3, 100), (32, 4, 256)])
def test_sample_fp64_multicomponent_and_sizes(ctx, ndim, ncomp, nbins):
    a, u = _params(ndim, ncomp, 100 + ndim)
    fams = [O.GAUSSIAN, O.OSCILLATORY, O.C0, O.PRODUCT_PEAK][:ncomp]
    edges = _random_grid(ndim, nbins, ndim)
    g = cg.genz(ndim, fams, a, u)
    n = 12345
    S1, S2, H = _gpu_sample(ctx, g, edges, 5, n, cg.FP64)
    p = O.Problem(ndim, fams, a, u, nbins=nbins, bits=52)
    oS1, oS2, oH = O.sample(p, edges, 5, n)
    np.testing.assert_allclose(S1, oS1, rtol=1e-12)
    np.testing.assert_allclose(S2, oS2, rtol=1e-12)
    scale = np.maximum(oH.max(axis=1, keepdims=True), 1e-300)
    assert np.all(np.abs(H - oH) <= 1e-12 * scale)


# ------------------------------------------------------------------ FP32 pass
@pytest.mark.parametrize("fam", FAMS)
@pytest.mark.parametrize("ndim,nbins,start,n", [(3, 50, 1, 20001), (8, 128, 77, 100000)])
def test_sample_fp32_matches_oracle(ctx, fam, ndim, nbins, start, n):
    a, u = _params(ndim, 1, 20 + fam)
    edges = _random_grid(ndim, nbins, 50 + fam)
    g = cg.genz(ndim, [fam], a, u)
    S1, S2, H = _gpu_sample(ctx, g, edges, start, n, 0)
    p = O.Problem(ndim, [fam], a, u, nbins=nbins, bits=23)
    check_fp32_pass(S1, S2, H, O.sample_bounds(p, edges, start, n), n)


def test_sample_fp32_const_is_exact(ctx):
    # f = 1, uniform power-of-two grid: J = 1, S1 = S2 = n, exact counts.
    ndim, N, n = 6, 64, 2 ** 16
    g = cg.genz(ndim, [cg.CONST], 1.0, 0.5)
    S1, S2, H = _gpu_sample(ctx, g, O.grid_uniform(ndim, N), 2 ** 16, n, 0)
    assert S1[0] == n and S2[0] == n
    assert np.all(H == n // N)


def test_sample_accumulates_and_zero_n_is_noop(ctx):
    ndim, N = 2, 16
    g = cg.genz(ndim, [cg.GAUSSIAN], 2.0, 0.5)
    e = torch.tensor(O.grid_uniform(ndim, N), device="cuda")
    S1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    S2 = torch.zeros_like(S1)
    H = torch.zeros((ndim, N), dtype=torch.float64, device="cuda")
    ctx.sample(g, N, e, 1, 0, cg.FP64, S1, S2, H)
    ctx.synchronize()
    assert S1.item() == 0.0
    ctx.sample(g, N, e, 1, 1000, cg.FP64, S1, S2, H)
    ctx.sample(g, N, e, 1001, 1000, cg.FP64, S1, S2, H)
    ctx.synchronize()
    p = O.Problem(ndim, [O.GAUSSIAN], np.full((1, ndim), 2.0), np.full((1, ndim), 0.5), nbins=N)
    oS1, _, _ = O.sample(p, O.grid_uniform(ndim, N), 1, 2000)
    assert S1.item() == pytest.approx(oS1[0], rel=1e-12)


# ------------------------------------------------------------------ refine
@pytest.mark.parametrize("ndim,nbins", [(1, 2), (3, 50), (8, 128), (32, 256)])
def test_refine_matches_oracle(ctx, ndim, nbins):
    rng = np.random.default_rng(nbins)
    edges = _random_grid(ndim, nbins, 3)
    H = rng.random((ndim, nbins)) ** 3
    H[0, : nbins // 3] = 0.0
    if ndim > 2:
        H[1] = 0.0          # all-zero axis keeps its grid
        H[2] = 1.0          # equal histogram keeps its grid
    e = torch.tensor(edges, device="cuda")
    h = torch.tensor(H, device="cuda")
    ctx.refine(ndim, nbins, h, e)
    ctx.synchronize()
    ref = O.refine(edges, H)
    assert np.max(np.abs(e.cpu().numpy() - ref)) <= 1e-14
    if ndim > 2:
        assert np.array_equal(e.cpu().numpy()[1:3], edges[1:3])


# ------------------------------------------------------------------ Vegas
def test_vegas_gaussian3d_fp64_matches_oracle(ctx):
    ndim, N, n = 3, 50, 10 ** 4
    g = cg.genz(ndim, [cg.GAUSSIAN], 5.0, 0.5)
    p = O.Problem(ndim, [O.GAUSSIAN], np.full((1, 3), 5.0), np.full((1, 3), 0.5), nbins=N)
    o = O.vegas(p, maxeval=10 * n, nstart=n)
    for flags in (cg.FP64, cg.FP64 | cg.PLAIN):
        r = ctx.vegas(g, flags=flags, maxeval=10 * n, nstart=n, nbins=N)
        assert (r.neval, r.fail) == (o.neval, o.fail)
        assert r.integral[0] == pytest.approx(o.integral[0], rel=1e-12)
        assert r.error[0] == pytest.approx(o.error[0], rel=1e-10)
        assert r.prob[0] == pytest.approx(o.prob[0], abs=1e-10)
    exact = (math.sqrt(math.pi) / 5 * math.erf(2.5)) ** 3
    assert abs(r.integral[0] - exact) < 3 * r.error[0]


def test_vegas_fp32_within_three_sigma_and_close_to_oracle(ctx):
    ndim, ncomp = 8, 4
    a, u = _params(ndim, ncomp, 7)
    fams = [O.OSCILLATORY, O.PRODUCT_PEAK, O.CORNER_PEAK, O.GAUSSIAN]
    g = cg.genz(ndim, fams, a, u)
    r = ctx.vegas(g, flags=0, maxeval=10 * 2 ** 15, nstart=2 ** 15, nbins=128)
    p = O.Problem(ndim, fams, a, u, nbins=128, bits=23)
    exact = p.exact()
    for c in range(ncomp):
        assert abs(r.integral[c] - exact[c]) < 3 * r.error[c] + 1e-7 * abs(exact[c])


def test_vegas_stops_on_accuracy_same_iteration_as_oracle(ctx):
    ndim = 4
    a, u = _params(ndim, 1, 3)
    g = cg.genz(ndim, [cg.GAUSSIAN], a, u)
    p = O.Problem(ndim, [O.GAUSSIAN], a, u, nbins=64)
    o = O.vegas(p, epsrel=2e-4, maxeval=10 ** 6, nstart=5000, nincrease=2500)
    r = ctx.vegas(g, epsrel=2e-4, flags=cg.FP64, maxeval=10 ** 6, nstart=5000, nincrease=2500, nbins=64)
    assert (r.neval, r.fail) == (o.neval, o.fail) and o.fail == 0
    assert r.integral[0] == pytest.approx(o.integral[0], rel=1e-12)


def test_vegas_const_exact(ctx):
    g = cg.genz(5, [cg.CONST], 1.0, 0.5)
    for flags in (0, cg.FP64):
        r = ctx.vegas(g, epsrel=1e-3, flags=flags, maxeval=10 ** 5, nstart=1024, nbins=64)
        assert r.integral[0] == 1.0 and r.error[0] == 0.0 and r.fail == 0 and r.neval == 1024


def test_vegas_nbatch_does_not_change_results(ctx):
    g = cg.genz(3, [cg.C0], 1.0, 0.4)
    r1 = ctx.vegas(g, flags=cg.FP64, maxeval=6 * 4000, nstart=4000, nbatch=100, nbins=32)
    r2 = ctx.vegas(g, flags=cg.FP64, maxeval=6 * 4000, nstart=4000, nbatch=100000, nbins=32)
    assert r1.integral[0] == pytest.approx(r2.integral[0], rel=1e-14)


def test_invalid_arguments_rejected(ctx):
    g = cg.genz(3, [cg.GAUSSIAN], 1.0, 0.5)
    with pytest.raises(cg.CubaGpuError) as ei:
        ctx.vegas(g, nbins=1)
    assert ei.value.code == cg.EINVAL
    with pytest.raises(cg.CubaGpuError):
        ctx.vegas(g, nstart=1)
    Y = torch.empty((3, 4), dtype=torch.int64, device="cuda")
    with pytest.raises(cg.CubaGpuError):
        ctx.sobol(3, 2 ** 52 - 2, 4, 52, Y)
    with pytest.raises(cg.CubaGpuError):
        ctx.sobol(3, 0, 4, 30, Y)
    bad = cg.genz(3, [9], 1.0, 0.5)
    with pytest.raises(cg.CubaGpuError):
        ctx.vegas(bad)


# ------------------------------------------------------------------ integral handle
def test_integral_handle_reruns_identically_and_matches_cv_vegas(ctx):
    ndim = 5
    a, u = _params(ndim, 2, 11)
    g = cg.genz(ndim, [cg.GAUSSIAN, cg.C0], a, u)
    sp = cg.spec(g, nbins=64, flags=cg.FP64, maxeval=6 * 8000, nstart=8000)
    I = ctx.integral(sp)
    I.reset()
    I.run()
    r1 = I.result()
    e1 = I.grid()
    I.reset()
    I.run()
    r2 = I.result()
    assert r1.iterations == 6 and r1.neval == 48000
    assert list(r1.integral)[:2] == pytest.approx(list(r2.integral)[:2], rel=1e-14)
    assert np.max(np.abs(I.grid() - e1)) <= 1e-15
    rv = ctx.vegas(g, flags=cg.FP64, maxeval=6 * 8000, nstart=8000, nbins=64)
    assert rv.integral[0] == pytest.approx(r1.integral[0], rel=1e-14)
    # the per-iteration log and final grid match the oracle's
    p = O.Problem(ndim, [O.GAUSSIAN, O.C0], a, u, nbins=64)
    o = O.vegas(p, maxeval=6 * 8000, nstart=8000)
    lI, lV = I.log(6)
    np.testing.assert_allclose(lI, o.iter_I, rtol=1e-12)
    np.testing.assert_allclose(lV, o.iter_var, rtol=1e-9)
    assert np.max(np.abs(I.grid() - o.edges)) <= 1e-13
    assert I.kernels_per_run() == 1 + 2 * 6
    I.close()


def test_fp32_iterations_with_grid_handed_to_oracle(ctx):
    # per-iteration parity of the FP32 path: each iteration's sums against
    # the oracle on the GPU's own grid, and the GPU refinement against the
    # oracle's refinement of the GPU histogram.
    ndim, N, n = 8, 128, 200000
    a, u = _params(ndim, 4, 21)
    fams = [O.OSCILLATORY, O.PRODUCT_PEAK, O.CORNER_PEAK, O.GAUSSIAN]
    g = cg.genz(ndim, fams, a, u)
    p = O.Problem(ndim, fams, a, u, nbins=N, bits=23)
    edges = O.grid_uniform(ndim, N)
    start = 1
    for it in range(4):
        S1, S2, H = _gpu_sample(ctx, g, edges, start, n, 0)
        check_fp32_pass(S1, S2, H, O.sample_bounds(p, edges, start, n, nthreads=8), n, what=it)
        e = torch.tensor(edges, device="cuda")
        h = torch.tensor(H, device="cuda")
        ctx.refine(ndim, N, h, e)
        ctx.synchronize()
        new = e.cpu().numpy()
        assert np.max(np.abs(new - O.refine(edges, H))) <= 1e-14
        edges = new
        start += n


@pytest.mark.parametrize("flags", [0, cg.JIT, cg.PSEUDO, cg.SCRAMBLE | cg.JIT])
@pytest.mark.parametrize("nbins", [128, 50])
def test_staged_grid_samples_like_the_fp64_grid(ctx, flags, nbins):
    # an integral's FP32 passes read the grid table its reset, refinement or
    # set_grid staged; a pass over the same grid that converts the FP64 edges
    # in the kernel (cv_sample) gives the same sums, up to the order of the
    # blocks' FP64 additions
    ndim, n, iters = 8, 200000, 4
    a, u = _params(ndim, 4, 33)
    g = cg.genz(ndim, [O.OSCILLATORY, O.PRODUCT_PEAK, O.CORNER_PEAK, O.GAUSSIAN], a, u)
    I = ctx.integral(cg.spec(g, nbins=nbins, maxeval=(iters + 1) * n, nstart=n, flags=flags))
    I.reset()
    start = 1
    for j in range(iters + 1):
        if j == iters:  # a grid set from the host
            I.set_grid(_random_grid(ndim, nbins, 5))
        edges = I.grid()
        I.step(1)
        Ij, Vj = I.log(j + 1)
        S1, S2, _ = _gpu_sample(ctx, g, edges, start, n, flags)
        for c in range(4):
            np.testing.assert_allclose(Ij[j, c], S1[c] / n, rtol=1e-12, atol=1e-15)
            var = (S2[c] / n - (S1[c] / n) ** 2) / (n - 1)
            np.testing.assert_allclose(Vj[j, c], var, rtol=1e-9)
        start += n
    I.close()


@pytest.mark.parametrize("flags", [0, cg.JIT, cg.PSEUDO, cg.SCRAMBLE])
@pytest.mark.parametrize("nbins", [128, 50, 16])
def test_sample_staged_equals_sample(ctx, flags, nbins):
    ndim, n = 6, 300000
    a, u = _params(ndim, 2, 8)
    g = cg.genz(ndim, [O.GAUSSIAN, O.OSCILLATORY], a, u)
    edges = _random_grid(ndim, nbins, 9)
    e = torch.tensor(edges, dtype=torch.float64, device="cuda")
    table = torch.empty((ndim, nbins, 2), dtype=torch.float32, device="cuda")
    ctx.stage_grid(ndim, nbins, flags, e, table)
    S1 = torch.zeros(2, dtype=torch.float64, device="cuda")
    S2, H = torch.zeros_like(S1), torch.zeros((ndim, nbins), dtype=torch.float64, device="cuda")
    ctx.sample_staged(g, nbins, table, 7, n, flags, S1, S2, H, seed=3)
    ctx.synchronize()
    rS1, rS2, rH = (t.cpu().numpy() for t in (S1, S2, H))
    S1, S2, H = (t.zero_() for t in (S1, S2, H))
    ctx.sample(g, nbins, e, 7, n, flags, S1, S2, H, seed=3)
    ctx.synchronize()
    np.testing.assert_allclose(rS1, S1.cpu().numpy(), rtol=1e-13)
    np.testing.assert_allclose(rS2, S2.cpu().numpy(), rtol=1e-13)
    # (warp-private FP32 histograms, for 2^L >= 32 bins and Sobol points, are
    # summed in a fixed order; the block histogram of the other layouts takes
    # FP32 shared-memory atomics in run-dependent order)
    private = nbins >= 32 and nbins & (nbins - 1) == 0 and not flags & cg.PSEUDO
    np.testing.assert_allclose(rH, H.cpu().numpy(), rtol=1e-12 if private else 1e-6, atol=1e-300)
    with pytest.raises(cg.CubaGpuError):
        ctx.sample_staged(g, nbins, table, 7, n, cg.FP64, S1, S2, H)
    with pytest.raises(cg.CubaGpuError):
        ctx.stage_grid(ndim, nbins, cg.FP64, e, table)


@pytest.mark.parametrize("nbins", [2, 16, 32, 64, 96, 256])
def test_sample_fp32_every_bin_layout(ctx, nbins):
    # power-of-two N >= 32 use the stratum-major shared-memory layout, other
    # N the plain one; both must give the oracle's sums and histogram.
    ndim, n = 5, 40001
    a, u = _params(ndim, 2, nbins)
    fams = [O.GAUSSIAN, O.DISCONTINUOUS]
    edges = _random_grid(ndim, nbins, nbins + 1)
    g = cg.genz(ndim, fams, a, u)
    S1, S2, H = _gpu_sample(ctx, g, edges, 3, n, 0)
    p = O.Problem(ndim, fams, a, u, nbins=nbins, bits=23)
    ob = O.sample_bounds(p, edges, 3, n)
    check_fp32_pass(S1, S2, H, ob, n)
    # the same points reach the same bins
    assert np.array_equal(H == 0, ob.H == 0)


@pytest.mark.parametrize("nbins", [32, 256])
def test_sample_fp32_const_counts_exact_permuted_layout(ctx, nbins):
    ndim, n = 3, 2 ** 15
    g = cg.genz(ndim, [cg.CONST], 1.0, 0.5)
    S1, S2, H = _gpu_sample(ctx, g, O.grid_uniform(ndim, nbins), 5 * n, n, 0)
    assert S1[0] == n and S2[0] == n and np.all(H == n // nbins)


def test_context_release_outlives_integral_handles():
    # destroying a context first releases the integrals still attached to it;
    # closing them afterwards is harmless.
    c = cg.Context(0)
    g = cg.genz(2, [cg.GAUSSIAN], 1.0, 0.5)
    I1 = c.integral(cg.spec(g, nbins=16, maxeval=4000, nstart=2000))
    I2 = c.integral(cg.spec(g, nbins=16, maxeval=4000, nstart=2000))
    I1.reset()
    I1.run()
    c.close()
    I1.close()
    I2.close()


# ------------------------------------------------------------------ run-time specialisation
def test_jit_specialised_kernel_matches_generic(ctx):
    ndim, N = 8, 128
    a, u = _params(ndim, 4, 33)
    fams = [O.OSCILLATORY, O.PRODUCT_PEAK, O.CORNER_PEAK, O.GAUSSIAN]
    g = cg.genz(ndim, fams, a, u)
    edges = _random_grid(ndim, N, 3)
    gen = _gpu_sample(ctx, g, edges, 1, 300000, 0)
    jit = _gpu_sample(ctx, g, edges, 1, 300000, cg.JIT)
    available, compiled = cg.jit_info()
    assert available and compiled >= 1
    for c in range(4):
        assert jit[0][c] == pytest.approx(gen[0][c], rel=1e-6, abs=1e-6 * math.sqrt(300000 * gen[1][c]))
        assert jit[1][c] == pytest.approx(gen[1][c], rel=1e-6)
    np.testing.assert_allclose(jit[2], gen[2], rtol=1e-5, atol=1e-5 * gen[2].max())
    # and both against the oracle on the same grid
    p = O.Problem(ndim, fams, a, u, nbins=N, bits=23)
    ob = O.sample_bounds(p, edges, 1, 300000, nthreads=8)
    check_fp32_pass(*jit, ob, 300000, what="jit")
    check_fp32_pass(*gen, ob, 300000, what="generic")


@pytest.mark.parametrize("ndim,fams,nbins", [(3, [O.DISCONTINUOUS], 50), (12, [O.C0, O.GAUSSIAN], 64),
                                             (1, [O.CORNER_PEAK], 32)])
def test_jit_vegas_runs_match_generic(ctx, ndim, fams, nbins):
    a, u = _params(ndim, len(fams), ndim)
    g = cg.genz(ndim, fams, a, u)
    kw = dict(maxeval=6 * 20000, nstart=20000, nbins=nbins)
    r0 = ctx.vegas(g, flags=0, **kw)
    r1 = ctx.vegas(g, flags=cg.JIT, **kw)
    assert r0.neval == r1.neval
    for c in range(len(fams)):
        assert abs(r1.integral[c] - r0.integral[c]) <= 2e-5 * abs(r0.integral[c]) + 1e-2 * r0.error[c]
