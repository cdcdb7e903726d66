"""Checkpoint/resume (the statefile of the Vegas prototype, Sect. 3.2.2)
and grid reuse (the role of gridno): an interrupted run resumed from a
saved state equals the uninterrupted run; a saved state only loads into
the same problem; a refined grid can seed another integral."""
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


def _spec(flags, maxeval=10 * 6000):
    a = np.array([[2.0, 3.0, 1.5, 2.5], [1.0, 1.0, 1.0, 1.0]])
    u = np.array([[0.3, 0.5, 0.7, 0.4], [0.5, 0.5, 0.5, 0.5]])
    g = cg.genz(4, [cg.GAUSSIAN, cg.C0], a, u)
    return cg.spec(g, nbins=64, flags=flags, maxeval=maxeval, nstart=6000, nincrease=2000)


# FP64: two runs of one problem agree to rounding (1e-14 run to run), so a
# resumed run must too.  FP32: the per-block bin histograms are summed with
# shared-memory atomics in a scheduling-dependent order, so two FP32 runs
# differ at FP32 rounding in their grids, which refinement feeds back; 1e-5
# bounds that drift over nine iterations.
@pytest.mark.parametrize("flags,rtol", [(cg.FP64, 1e-13), (0, 1e-5)])
def test_resume_from_saved_state_equals_uninterrupted_run(ctx, tmp_path, flags, rtol):
    full = ctx.integral(_spec(flags, maxeval=10 ** 6))
    full.reset()
    full.step(9)
    ref = full.result()
    a = ctx.integral(_spec(flags, maxeval=10 ** 6))
    a.reset()
    a.step(4)
    path = str(tmp_path / "vegas.state")
    a.save(path)
    a.close()
    b = ctx.integral(_spec(flags, maxeval=10 ** 6))
    b.load(path)
    b.step(5)
    res = b.result()
    assert (res.iterations, res.neval) == (ref.iterations, ref.neval) == (9, sum(6000 + 2000 * j for j in range(9)))
    np.testing.assert_allclose(list(res.integral)[:2], list(ref.integral)[:2], rtol=rtol)
    np.testing.assert_allclose(list(res.error)[:2], list(ref.error)[:2], rtol=100 * rtol)
    if flags == cg.FP64:
        # and the FP64 run equals the oracle's nine iterations
        p = O.Problem(4, [O.GAUSSIAN, O.C0], np.array([[2.0, 3.0, 1.5, 2.5], [1.0] * 4]),
                      np.array([[0.3, 0.5, 0.7, 0.4], [0.5] * 4]), nbins=64)
        o = O.vegas(p, maxeval=sum(6000 + 2000 * j for j in range(9)), nstart=6000, nincrease=2000)
        np.testing.assert_allclose(list(res.integral)[:2], o.integral, rtol=1e-12)
    b.close()
    full.close()


def test_state_of_another_problem_is_refused(ctx, tmp_path):
    a = ctx.integral(_spec(cg.FP64))
    a.reset()
    a.step(2)
    path = str(tmp_path / "s")
    a.save(path)
    other = ctx.integral(_spec(0))
    with pytest.raises(cg.CubaGpuError):
        other.load(path)
    with pytest.raises(cg.CubaGpuError):
        other.load(str(tmp_path / "missing"))
    a.close()
    other.close()


def test_grid_reuse_seeds_a_new_integral(ctx):
    sp = _spec(cg.FP64, maxeval=8 * 6000)
    sp.nincrease = 0
    first = ctx.integral(sp)
    first.reset()
    first.run()
    grid = first.grid()
    # a warm start from the refined grid: the first iteration already has
    # the small variance of an adapted grid
    warm = ctx.integral(sp)
    warm.reset()
    warm.set_grid(grid)
    warm.step(1)
    cold = ctx.integral(sp)
    cold.reset()
    cold.step(1)
    assert warm.log(1)[1][0, 0] < 0.5 * cold.log(1)[1][0, 0]
    bad = grid.copy()
    bad[0, 5] = bad[0, 4]
    with pytest.raises(cg.CubaGpuError):
        warm.set_grid(bad)
    # the warm-started run equals the oracle started from the same grid
    warm.reset()
    warm.set_grid(grid)
    warm.run()
    r = warm.result()
    p = O.Problem(4, [O.GAUSSIAN, O.C0], np.array([[2.0, 3.0, 1.5, 2.5], [1.0] * 4]),
                  np.array([[0.3, 0.5, 0.7, 0.4], [0.5] * 4]), nbins=64)
    o = O.vegas(p, maxeval=8 * 6000, nstart=6000, edges=grid)
    assert r.iterations == 8
    np.testing.assert_allclose(list(r.integral)[:2], o.integral, rtol=1e-12)
    np.testing.assert_allclose(warm.log(8)[0], o.iter_I[:8], rtol=1e-12)
    assert np.max(np.abs(warm.grid() - o.edges)) <= 1e-13
    for I in (first, warm, cold):
        I.close()
