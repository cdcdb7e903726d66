"""GPU tests of the materialised-sample mode (cv_vegas_cb): the integrand
contract of Sect. 3.2.1-3.2.2 on the device -- up to nvec points per call,
the actual count passed, -999 aborts -- in both layouts, against the fused
path and the FP64 oracle."""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle as O
from tests.tolerances import check_fp32_iteration

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


def _genz(ndim=5, seed=3):
    rng = np.random.default_rng(seed)
    a = 0.5 + rng.random((2, ndim))
    u = rng.random((2, ndim))
    return cg.genz(ndim, [cg.GAUSSIAN, cg.PRODUCT_PEAK], a, u), a, u


@pytest.mark.parametrize("aos", [False, True])
def test_builtin_integrand_fp64_matches_oracle_and_fused(ctx, aos):
    g, a, u = _genz()
    flags = cg.FP64 | (cg.AOS if aos else 0)
    ud = cg.GenzCallbackData(g, flags)
    kw = dict(maxeval=6 * 12000, nstart=12000, nbins=50)
    r = ctx.vegas_cb(cg.builtin_integrand(), 5, 2, userdata=ud, nvec=5000, flags=flags, **kw)
    fused = ctx.vegas(g, flags=cg.FP64, **kw)
    o = O.vegas(O.Problem(5, [O.GAUSSIAN, O.PRODUCT_PEAK], a, u, nbins=50), maxeval=kw["maxeval"],
                nstart=kw["nstart"])
    assert (r.neval, r.fail) == (o.neval, o.fail)
    np.testing.assert_allclose(r.integral, o.integral, rtol=1e-12)
    np.testing.assert_allclose(r.integral, fused.integral, rtol=1e-12)
    np.testing.assert_allclose(r.error, o.error, rtol=1e-10)


def test_builtin_integrand_fp32_close_to_fused(ctx):
    g, a, u = _genz(seed=4)
    ud = cg.GenzCallbackData(g, 0)
    kw = dict(maxeval=5 * 20000, nstart=20000, nbins=64)
    r = ctx.vegas_cb(cg.builtin_integrand(), 5, 2, userdata=ud, nvec=1 << 20, flags=0, **kw)
    fused = ctx.vegas(g, flags=0, **kw)
    for c in range(2):
        assert abs(r.integral[c] - fused.integral[c]) <= 2e-5 * abs(fused.integral[c]) + 1e-2 * fused.error[c]


# One FP32 iteration on the uniform grid through the materialised passes
# (points written, the library's integrand, values read back) against the
# oracle's pass: I_1 and var_1 (error^2 of a one-iteration run) within the
# FP32 bounds.  Tiles of 3333 points start at unaligned indices (the store
# pass's shifted warps, ragged last tiles); 64 and 128 bins take the
# dimension-major power-of-two kernels, 50 bins the general pass; scrambled
# points too; the library's integrand generic or specialised at run time.
@pytest.mark.parametrize("jit", [0, cg.JIT], ids=["generic", "jit"])
@pytest.mark.parametrize("gen", ["sobol", "scrambled"])
@pytest.mark.parametrize("nbins", [64, 128, 50])
@pytest.mark.parametrize("nvec", [3333, 1 << 16])
def test_materialised_fp32_pass_matches_oracle(ctx, nvec, nbins, gen, jit):
    ndim, fams = 8, [O.GAUSSIAN, O.PRODUCT_PEAK, O.OSCILLATORY, O.C0]
    rng = np.random.default_rng(17 + nbins)
    a = rng.uniform(0.5, 1.5, (4, ndim))
    u = rng.uniform(0.1, 0.9, (4, ndim))
    n = 100003
    flags, seed = (cg.SCRAMBLE, 11) if gen == "scrambled" else (0, 0)
    g = cg.genz(ndim, fams, a, u)
    r = ctx.vegas_cb(cg.builtin_integrand(), ndim, 4, userdata=cg.GenzCallbackData(g, jit), nvec=nvec,
                     flags=flags, seed=seed, maxeval=n, nstart=n, nbins=nbins)
    assert (r.neval, r.fail) == (n, 1)
    p = O.Problem(ndim, fams, a, u, nbins=nbins, bits=23, gen=O.SCRAMBLED if flags else O.SOBOL, seed=seed)
    ob = O.sample_bounds(p, O.grid_uniform(ndim, nbins), 1, n, nthreads=os.cpu_count() or 1)
    check_fp32_iteration(r.integral, r.error ** 2, ob, n, what=(nvec, nbins, gen))


# The dimension-major FP32 kernels above 16 dimensions (their group steps
# take a run-time word), one iteration against the oracle's pass.
@pytest.mark.parametrize("ndim", [17, 24, 30])
def test_materialised_fp32_high_dimensions_match_oracle(ctx, ndim):
    fams = [O.GAUSSIAN, O.C0]
    rng = np.random.default_rng(ndim)
    a = rng.uniform(0.2, 0.6, (2, ndim))
    u = rng.uniform(0.1, 0.9, (2, ndim))
    n = 150001
    g = cg.genz(ndim, fams, a, u)
    r = ctx.vegas_cb(cg.builtin_integrand(), ndim, 2, userdata=cg.GenzCallbackData(g, cg.JIT), nvec=40000,
                     flags=0, maxeval=n, nstart=n, nbins=64)
    assert (r.neval, r.fail) == (n, 1)
    p = O.Problem(ndim, fams, a, u, nbins=64, bits=23)
    ob = O.sample_bounds(p, O.grid_uniform(ndim, 64), 1, n, nthreads=os.cpu_count() or 1)
    check_fp32_iteration(r.integral, r.error ** 2, ob, n, what=("highdim", ndim))


# The point-major layout in FP32 (the paper's x[j*ndim + d]; the general
# materialised passes and the library's general integrand), one iteration
# against the oracle's pass as above.
@pytest.mark.parametrize("nbins", [64, 50])
def test_materialised_fp32_point_major_pass_matches_oracle(ctx, nbins):
    ndim, fams = 7, [O.PRODUCT_PEAK, O.GAUSSIAN, O.C0]
    rng = np.random.default_rng(41 + nbins)
    a = rng.uniform(0.5, 1.5, (3, ndim))
    u = rng.uniform(0.1, 0.9, (3, ndim))
    n = 70001
    g = cg.genz(ndim, fams, a, u)
    r = ctx.vegas_cb(cg.builtin_integrand(), ndim, 3, userdata=cg.GenzCallbackData(g, cg.AOS), nvec=4099,
                     flags=cg.AOS, maxeval=n, nstart=n, nbins=nbins)
    assert (r.neval, r.fail) == (n, 1)
    p = O.Problem(ndim, fams, a, u, nbins=nbins, bits=23)
    ob = O.sample_bounds(p, O.grid_uniform(ndim, nbins), 1, n, nthreads=os.cpu_count() or 1)
    check_fp32_iteration(r.integral, r.error ** 2, ob, n, what=("aos", nbins))


def test_tiles_do_not_change_results(ctx):
    g, _, _ = _genz(seed=5)
    ud = cg.GenzCallbackData(g, cg.FP64)
    kw = dict(flags=cg.FP64, maxeval=4 * 10000, nstart=10000, nbins=32)
    one = ctx.vegas_cb(cg.builtin_integrand(), 5, 2, userdata=ud, nvec=10000, **kw)
    many = ctx.vegas_cb(cg.builtin_integrand(), 5, 2, userdata=ud, nvec=777, **kw)
    np.testing.assert_allclose(one.integral, many.integral, rtol=1e-13)


# The accumulate passes reduce through per-block partials in a fixed order
# (no floating-point atomics): the same run twice gives the same bits, with
# one tile per iteration (partials summed by the combination) and with many
# (each pass adds its own), in the FP32 power-of-two kernels and in FP64
# and the point-major layout's general pass (warp-private histograms for
# N = 2^L >= 32; other bin counts update one block copy with shared-memory
# atomics).
@pytest.mark.parametrize("flags,nbins", [(0, 128), (cg.JIT, 64), (cg.FP64, 32), (cg.FP64 | cg.AOS, 64)],
                         ids=["f32-128", "f32-jit-64", "f64-32", "f64-aos-64"])
@pytest.mark.parametrize("nvec", [1 << 17, 7777], ids=["one-tile", "tiles"])
def test_materialised_runs_agree_bit_for_bit(ctx, flags, nbins, nvec):
    g, _, _ = _genz(ndim=6, seed=9)
    kw = dict(flags=flags & ~cg.JIT, maxeval=5 * 30000, nstart=30000, nincrease=10000, nbins=nbins)
    ud = cg.GenzCallbackData(g, flags)
    r = [ctx.vegas_cb(cg.builtin_integrand(), 6, 2, userdata=ud, nvec=nvec, **kw) for _ in range(3)]
    for x in r[1:]:
        assert (x.neval, x.fail) == (r[0].neval, r[0].fail)
        for key in ("integral", "error", "prob"):
            assert np.array_equal(np.asarray(getattr(x, key)).view(np.uint64),
                                  np.asarray(getattr(r[0], key)).view(np.uint64)), (key, flags, nbins, nvec)


# Tiles far smaller than a warp's 32 points (1, 7 and 31 points per call):
# every tile's accumulate pass takes the edge path, adds its own partial
# rows, and the iteration still equals the oracle's pass.
@pytest.mark.parametrize("flags,nbins", [(0, 64), (cg.FP64, 32), (0, 50)], ids=["f32-64", "f64-32", "f32-50"])
@pytest.mark.parametrize("nvec", [1, 7, 31])
def test_tiny_tiles_match_oracle(ctx, flags, nbins, nvec):
    ndim, fams = 3, [O.GAUSSIAN, O.C0]
    rng = np.random.default_rng(5 + nvec)
    a = rng.uniform(0.5, 1.5, (2, ndim))
    u = rng.uniform(0.1, 0.9, (2, ndim))
    n = 403
    g = cg.genz(ndim, fams, a, u)
    r = ctx.vegas_cb(cg.builtin_integrand(), ndim, 2, userdata=cg.GenzCallbackData(g, flags & cg.FP64),
                     nvec=nvec, flags=flags, maxeval=n, nstart=n, nbins=nbins)
    assert (r.neval, r.fail) == (n, 1)
    if flags & cg.FP64:
        o = O.vegas(O.Problem(ndim, fams, a, u, nbins=nbins), maxeval=n, nstart=n)
        np.testing.assert_allclose(r.integral, o.integral, rtol=1e-12)
        np.testing.assert_allclose(r.error, o.error, rtol=1e-10)
    else:
        p = O.Problem(ndim, fams, a, u, nbins=nbins, bits=23)
        ob = O.sample_bounds(p, O.grid_uniform(ndim, nbins), 1, n, nthreads=1)
        check_fp32_iteration(r.integral, r.error ** 2, ob, n, what=("tiny", nvec, nbins))


def test_torch_integrand_and_nvec_contract(ctx):
    # a user integrand written with torch on the device buffers
    ndim = 4
    a = torch.tensor([3.0, 2.0, 2.5, 1.5], device="cuda")
    u = torch.tensor([0.5, 0.4, 0.6, 0.3], device="cuda")
    seen = []

    def gauss(x, f, nvec, stream):
        seen.append(nvec)
        f[0].copy_(torch.exp(-(((x - u[:, None]) * a[:, None]) ** 2).sum(0)))
        return 0

    r = ctx.vegas_cb(gauss, ndim, 1, nvec=3000, flags=0, maxeval=5 * 8000, nstart=8000, nbins=32)
    assert max(seen) <= 3000 and sum(seen) == 5 * 8000
    exact = O.genz_exact(O.GAUSSIAN, a.cpu().numpy(), u.cpu().numpy())
    assert abs(r.integral[0] - exact) < 3 * r.error[0] + 1e-6 * exact
    g = cg.genz(ndim, [cg.GAUSSIAN], a.cpu().numpy(), u.cpu().numpy())
    ref = ctx.vegas_cb(cg.builtin_integrand(), ndim, 1, userdata=cg.GenzCallbackData(g, 0), nvec=3000,
                       flags=0, maxeval=5 * 8000, nstart=8000, nbins=32)
    assert r.integral[0] == pytest.approx(ref.integral[0], rel=1e-5)


def test_integrand_abort(ctx):
    calls = []

    def abort_second(x, f, nvec, stream):
        calls.append(nvec)
        f.fill_(1.0)
        return -999 if len(calls) == 2 else 0

    r = ctx.vegas_cb(abort_second, 3, 1, nvec=1000, flags=0, maxeval=10 * 5000, nstart=5000, nbins=16)
    assert r.fail == -999 and len(calls) == 2


def test_aos_layout_seen_by_integrand(ctx):
    shapes = []

    def rec(x, f, nvec, stream):
        shapes.append(tuple(x.shape))
        f[:, 0].copy_(x.sum(1))
        return 0

    r = ctx.vegas_cb(rec, 3, 1, nvec=2048, flags=cg.AOS | cg.FP64, maxeval=2 * 4096, nstart=4096,
                     nbins=16)
    assert shapes[0] == (2048, 3)
    # integral of x1 + x2 + x3 over the unit cube
    assert r.integral[0] == pytest.approx(1.5, rel=1e-4)


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
@pytest.mark.parametrize("flags", [0, cg.FP64])
def test_nonfinite_integrand_value_stops_the_run(ctx, bad, flags):
    # the integrand contract (Sect. 3.2.1-3.2.2) on the device: a value that
    # is not finite, written by the caller's integrand into one tile of the
    # third iteration, is detected in that iteration's combination; the run
    # stops there with fail = 1 (not "accuracy reached", whatever the goal)
    # and the call reports CV_ENONFINITE
    n, nvec = 6000, 2500
    calls = []

    def poisoned(x, f, nvec_, stream):
        calls.append(nvec_)
        f[0].copy_(x.sum(0))
        if len(calls) == 8:  # iterations of 3 tiles each: the 2nd tile of the 3rd
            f[0, 17] = bad
        return 0

    # (mineval: the goal alone could not stop the run before iteration 5)
    r = ctx.vegas_cb(poisoned, 3, 1, nvec=nvec, flags=flags, epsrel=1e-1, mineval=5 * n, maxeval=10 * n,
                     nstart=n, nbins=16)
    assert r.code == cg.ENONFINITE and r.fail == 1
    assert r.neval == 3 * n and sum(calls) == 3 * n
    assert not math.isfinite(r.integral[0]) or not math.isfinite(r.error[0])
    # the same integrand without the bad value converges on the goal
    ok = ctx.vegas_cb(lambda x, f, m, s: (f[0].copy_(x.sum(0)), 0)[1], 3, 1, nvec=nvec, flags=flags,
                      epsrel=1e-1, mineval=5 * n, maxeval=10 * n, nstart=n, nbins=16)
    assert ok.code == 0 and ok.fail == 0 and ok.neval == 5 * n
    assert ok.integral[0] == pytest.approx(1.5, rel=1e-3)
