"""GPU Suave against the oracle's Suave through the C ABI.

FP64: the same decisions (regions, evaluations, boxes) and the integral
within 1e-10 (the region sums differ from the oracle's only in summation
order; the decisions are taken from FP64 values on both sides).  FP32 (the
batched passes): the FP64 run's decisions, its integral within 1e-5.  FP32
and the other generators: the closed form within 4 sigma.
"""
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


CASES = [(3, O.GAUSSIAN, [6.0, 4.0, 5.0], [0.3, 0.6, 0.5], 1),
         (3, O.GAUSSIAN, [6.0, 4.0, 5.0], [0.3, 0.6, 0.5], 8),
         (2, O.PRODUCT_PEAK, [4.0, 3.0], [0.4, 0.7], 4),
         (4, O.CORNER_PEAK, [1.0, 2.0, 0.5, 1.5], [0.5] * 4, 3)]


@pytest.mark.parametrize("ndim,fam,a,u,width", CASES)
def test_fp64_matches_oracle(ctx, ndim, fam, a, u, width):
    a, u = np.array([a]), np.array([u])
    kw = dict(epsrel=2e-4, maxeval=200000, nnew=2000, width=width, max_regions=512)
    g = cg.genz(ndim, [fam], a, u)
    r = ctx.suave(g, nbins=16, flags=cg.FP64, **kw)
    o = O.suave(O.Problem(ndim, [fam], a, u, nbins=16), **kw)
    assert (r.nregions, r.neval, r.fail) == (o.nregions, o.neval, o.fail)
    np.testing.assert_allclose(r.boxes, o.boxes, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.integral, o.integral, rtol=1e-10)
    np.testing.assert_allclose(r.error, o.error, rtol=1e-8)


@pytest.mark.parametrize("flag,gen", [(cg.SCRAMBLE, O.SCRAMBLED), (cg.PSEUDO, O.PSEUDO)])
def test_fp64_generators_match_oracle(ctx, flag, gen):
    a, u = np.array([[5.0, 3.0, 4.0]]), np.array([[0.4, 0.5, 0.6]])
    kw = dict(epsrel=3e-4, maxeval=100000, nnew=2000, width=4, max_regions=256)
    r = ctx.suave(cg.genz(3, [O.GAUSSIAN], a, u), nbins=16, flags=cg.FP64 | flag, seed=9, **kw)
    o = O.suave(O.Problem(3, [O.GAUSSIAN], a, u, nbins=16, gen=gen, seed=9), **kw)
    assert (r.nregions, r.neval) == (o.nregions, o.neval)
    np.testing.assert_allclose(r.integral, o.integral, rtol=1e-10)


@pytest.mark.parametrize("flags", [0, cg.JIT])
def test_fp32_meets_the_closed_form(ctx, flags):
    a, u = np.array([[6.0, 4.0, 5.0, 3.0]]), np.array([[0.3, 0.6, 0.5, 0.4]])
    r = ctx.suave(cg.genz(4, [O.GAUSSIAN], a, u), nbins=32, flags=flags, epsrel=1e-4, maxeval=2000000,
                  nnew=20000, width=16, max_regions=1024)
    exact = O.genz_exact(O.GAUSSIAN, a[0], u[0])
    assert r.nregions > 8
    assert abs(r.integral[0] - exact) < 3 * r.error[0] + 1e-6 * exact
    vol = np.prod(r.boxes[:, :, 1] - r.boxes[:, :, 0], axis=1)
    assert abs(vol.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("ndim,fam,a,u,width", CASES)
@pytest.mark.parametrize("nbins", [16, 32])
def test_fp32_takes_the_fp64_decisions(ctx, ndim, fam, a, u, width, nbins):
    # FP32 passes (one batched sampling launch over all regions of a pass)
    # reach the FP64 run's regions and evaluations; boxes and the integral
    # agree to the FP32 sums' rounding
    a, u = np.array([a]), np.array([u])
    kw = dict(nbins=nbins, epsrel=2e-4, maxeval=400000, nnew=4000, width=width, max_regions=512)
    g = cg.genz(ndim, [fam], a, u)
    r64 = ctx.suave(g, flags=cg.FP64, **kw)
    r32 = ctx.suave(g, flags=0, **kw)
    assert (r32.nregions, r32.neval, r32.fail) == (r64.nregions, r64.neval, r64.fail)
    np.testing.assert_allclose(r32.boxes, r64.boxes, rtol=0, atol=1e-5)
    np.testing.assert_allclose(r32.integral, r64.integral, rtol=1e-5)
    np.testing.assert_allclose(r32.error, r64.error, rtol=1e-3)


@pytest.mark.parametrize("flags", [cg.SCRAMBLE, cg.PSEUDO])
def test_fp32_generators_meet_the_closed_form(ctx, flags):
    # scrambled points take the batched passes, pseudo-random points one
    # launch per region
    a, u = np.array([[6.0, 4.0, 5.0, 3.0, 5.5]]), np.array([[0.3, 0.6, 0.5, 0.4, 0.55]])
    r = ctx.suave(cg.genz(5, [O.GAUSSIAN], a, u), nbins=32, flags=flags, seed=3, epsrel=1e-4,
                  maxeval=4000000, nnew=1 << 15, width=32, max_regions=2048)
    exact = O.genz_exact(O.GAUSSIAN, a[0], u[0])
    assert r.nregions > 32
    assert abs(r.integral[0] - exact) < 3 * r.error[0] + 1e-6 * exact


def test_bad_arguments(ctx):
    g = cg.genz(2, [O.GAUSSIAN], 1.0, 0.5)
    for kw in (dict(nbins=15), dict(nnew=1), dict(width=0), dict(flatness=0.0), dict(maxeval=10, nnew=100)):
        args = dict(nbins=16, maxeval=10000, nnew=1000)
        args.update(kw)
        with pytest.raises(cg.CubaGpuError):
            ctx.suave(g, **args)
