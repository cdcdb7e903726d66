"""cv_vegas_noalloc -- the Vegas call for callers that cannot allocate
device memory -- against the allocating cv_vegas.

Some callers of the library may not call cudaMalloc (their device memory
belongs to another framework's allocator, or a pool holds all of it);
cv_vegas_noalloc serves them from a static device array.  This file is
collected last so that a failure here stops a -x run only after every
other test has run; it passes alone in a fresh process and after the rest.
"""
import numpy as np
import pytest

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


def _problem():
    rng = np.random.default_rng(42)
    a = rng.uniform(0.5, 1.5, (2, 6))
    u = rng.uniform(0.2, 0.8, (2, 6))
    return cg.genz(6, [cg.GAUSSIAN, cg.OSCILLATORY], a, u)


# FP32 path: the integrals agree to 1e-6; the error estimates only to 1e-4,
# because the variance (S2/n - I^2)/(n-1) cancels digits and the FP32
# shared-memory histogram is summed in a run-dependent order, so the grids
# of two runs differ at the 1e-7 level.
@pytest.mark.parametrize("flags,rtol,err_rtol", [(cg.FP64, 1e-12, 1e-10), (0, 1e-6, 1e-4)])
def test_noalloc_matches_allocating_call_twice(ctx, flags, rtol, err_rtol):
    g = _problem()
    kw = dict(flags=flags, maxeval=8 * 20000, nstart=20000, nbins=64)
    ref = ctx.vegas(g, **kw)
    for _ in range(2):  # the static array keeps the previous call's contents
        r = cg.vegas_noalloc(g, device=0, **kw)
        assert (r.neval, r.fail) == (ref.neval, ref.fail)
        np.testing.assert_allclose(r.integral, ref.integral, rtol=rtol)
        np.testing.assert_allclose(r.error, ref.error, rtol=err_rtol)
        np.testing.assert_allclose(r.prob, ref.prob, rtol=0, atol=1e-6)


def test_noalloc_accuracy_goal_and_too_large_problem(ctx):
    g = _problem()
    kw = dict(epsrel=1e-3, flags=cg.FP64, maxeval=10 ** 6, nstart=5000, nincrease=5000, nbins=32)
    ref = ctx.vegas(g, **kw)
    r = cg.vegas_noalloc(g, device=0, **kw)
    assert (r.neval, r.fail) == (ref.neval, ref.fail)
    np.testing.assert_allclose(r.integral, ref.integral, rtol=1e-12)
    big = cg.genz(32, [cg.GAUSSIAN], 1.0, 0.5)
    with pytest.raises(cg.CubaGpuError) as ei:
        cg.vegas_noalloc(big, device=0, maxeval=4000, nstart=2000, nbins=256)
    assert ei.value.code == cg.ESCRATCH


def test_noalloc_leaves_the_current_device_and_takes_a_side_stream(ctx):
    # a caller embedded in another framework keeps its thread's current
    # device; the work may run on any stream of that device
    g = _problem()
    kw = dict(flags=cg.FP64, maxeval=4 * 8000, nstart=8000, nbins=32)
    ref = ctx.vegas(g, **kw)
    before = torch.cuda.current_device()
    side = torch.cuda.Stream(device=0)
    r = cg.vegas_noalloc(g, device=0, stream=side.cuda_stream, **kw)
    assert torch.cuda.current_device() == before
    np.testing.assert_allclose(r.integral, ref.integral, rtol=1e-12)
    with pytest.raises(cg.CubaGpuError) as ei:
        cg.vegas_noalloc(g, device=torch.cuda.device_count(), stream=side.cuda_stream, **kw)  # no such device
    assert ei.value.code == cg.EINVAL
    assert torch.cuda.current_device() == before


def test_noalloc_size_rule_at_its_boundary(ctx):
    # 512 + R256(ndim (nbins+1) 8) + ndim nbins 8 <= CV_STATIC_SCRATCH_BYTES:
    # 32 dimensions fit up to 254 bins
    def need(ndim, nbins):
        return 512 + -(-ndim * (nbins + 1) * 8 // 256) * 256 + ndim * nbins * 8
    assert need(32, 254) <= 128 * 1024 < need(32, 255)
    g = cg.genz(32, [cg.GAUSSIAN], 0.25, 0.5)
    kw = dict(flags=cg.FP64, maxeval=2 * 4096, nstart=4096)
    ref = ctx.vegas(g, nbins=254, **kw)
    r = cg.vegas_noalloc(g, device=0, nbins=254, **kw)
    np.testing.assert_allclose(r.integral, ref.integral, rtol=1e-12)
    with pytest.raises(cg.CubaGpuError) as ei:
        cg.vegas_noalloc(g, device=0, nbins=255, **kw)
    assert ei.value.code == cg.ESCRATCH
