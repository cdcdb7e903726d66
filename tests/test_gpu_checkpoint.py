"""Checkpoint/resume (the statefile of the Vegas prototype, Sect. 3.2.2)
and grid reuse (the role of gridno): an interrupted run resumed from a
saved state equals the uninterrupted run; a saved state only loads into
the same problem; a refined grid can seed another integral."""
import ctypes

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


# Every sum of an integral's pass is reduced in a fixed order (per-warp
# histograms for Sobol points and 2^L >= 32 bins, per-block partials added in
# block order), so a run is reproducible bit for bit and a resumed run is
# the uninterrupted run, bit for bit, in FP64 and FP32.
@pytest.mark.parametrize("flags", [cg.FP64, 0, cg.JIT])
def test_resume_from_saved_state_equals_uninterrupted_run(ctx, tmp_path, flags):
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
    # the saved file passes the host-side checks load makes
    assert cg.check_state_file(_spec(flags, maxeval=10 ** 6), path) == (True, "")
    b = ctx.integral(_spec(flags, maxeval=10 ** 6))
    b.load(path)
    b.step(5)
    res = b.result()
    assert (res.iterations, res.neval) == (ref.iterations, ref.neval) == (9, sum(6000 + 2000 * j for j in range(9)))
    assert list(res.integral)[:2] == list(ref.integral)[:2]
    assert list(res.error)[:2] == list(ref.error)[:2]
    assert list(res.prob)[:2] == list(ref.prob)[:2]
    assert np.array_equal(b.grid(), full.grid())
    if flags == cg.FP64:
        # and the FP64 run equals the oracle's nine iterations
        p = O.Problem(4, [O.GAUSSIAN, O.C0], np.array([[2.0, 3.0, 1.5, 2.5], [1.0] * 4]),
                      np.array([[0.3, 0.5, 0.7, 0.4], [0.5] * 4]), nbins=64)
        o = O.vegas(p, maxeval=sum(6000 + 2000 * j for j in range(9)), nstart=6000, nincrease=2000)
        np.testing.assert_allclose(list(res.integral)[:2], o.integral, rtol=1e-12)
    b.close()
    full.close()


@pytest.mark.parametrize("flags", [cg.FP64, 0, cg.JIT, cg.SCRAMBLE])
def test_two_runs_agree_bit_for_bit(ctx, flags):
    # the same run twice, and the one-shot call, give identical bits; so do
    # two standalone passes accumulated into fresh buffers
    sp = _spec(flags, maxeval=12 * 6000)
    sp.seed = 5
    r = []
    for _ in range(2):
        I = ctx.integral(sp)
        I.reset()
        I.run()
        r.append((I.result(), I.grid()))
        I.close()
    assert list(r[0][0].integral) == list(r[1][0].integral)
    assert list(r[0][0].error) == list(r[1][0].error)
    assert np.array_equal(r[0][1], r[1][1])
    one = ctx.vegas(sp.g, flags=flags, seed=5, maxeval=sp.maxeval, nstart=sp.nstart, nincrease=sp.nincrease,
                    nbins=sp.nbins)
    assert list(one.integral) == list(r[0][0].integral)[:2]
    e = torch.tensor(r[0][1], dtype=torch.float64, device="cuda")
    outs = []
    for _ in range(2):
        S1 = torch.zeros(2, dtype=torch.float64, device="cuda")
        S2, H = torch.zeros_like(S1), torch.zeros((4, 64), dtype=torch.float64, device="cuda")
        ctx.sample(sp.g, 64, e, 12345, 300001, flags, S1, S2, H, seed=5)
        ctx.synchronize()
        outs.append([t.cpu().numpy() for t in (S1, S2, H)])
    for x, y in zip(*outs):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("epsrel", [0.0, 2e-3], ids=["fixed", "goal"])
@pytest.mark.parametrize("flags", [0, cg.JIT, cg.FP64])
def test_repeated_vegas_calls_give_the_same_bits(ctx, flags, epsrel):
    # cv_vegas keeps the last call's integral: a repeat of the same problem
    # replays its iterations from a captured graph (the second call captures,
    # later calls replay), another problem in between starts afresh, and the
    # kernel timer forces direct launches: every path gives the same bits
    # (80 iterations: the graph holds 32, so a run is three replays, and with
    # an accuracy goal the device's stop is polled between them)
    sp = cg.spec(_spec(flags).g, nbins=64, flags=flags, maxeval=80 * 2000, nstart=2000)
    other = _spec(flags, maxeval=3 * 6000)
    kw = dict(flags=flags, maxeval=sp.maxeval, nstart=sp.nstart, nincrease=sp.nincrease, nbins=sp.nbins,
              epsrel=epsrel)

    def bits(r):
        return [np.float64(v).view(np.uint64) for key in ("integral", "error", "prob") for v in getattr(r, key)]

    first = ctx.vegas(sp.g, **kw)
    runs = [ctx.vegas(sp.g, **kw) for _ in range(3)]
    o = ctx.vegas(other.g, flags=flags, maxeval=other.maxeval, nstart=other.nstart,
                  nincrease=other.nincrease, nbins=other.nbins)
    assert o.fail == 1 and 0 < o.neval <= other.maxeval
    runs.append(ctx.vegas(sp.g, **kw))
    ctx.kernel_timer(True)
    runs.append(ctx.vegas(sp.g, **kw))
    ctx.kernel_timer(False)
    runs.append(ctx.vegas(sp.g, **kw))
    if epsrel:
        assert first.neval <= sp.maxeval and (first.fail == 0) == (first.neval < sp.maxeval)
    for r in runs:
        assert (r.neval, r.fail) == (first.neval, first.fail)
        assert bits(r) == bits(first)


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
    # a damaged copy (the next Sobol index moved by one) is refused before
    # it reaches the device, and the integral it was meant for still runs
    from tests.test_state_file import Header
    data = bytearray(open(path, "rb").read())
    off = ctypes.sizeof(Header)
    data[off:off + 8] = (int.from_bytes(data[off:off + 8], "little") + 1).to_bytes(8, "little")
    bad = str(tmp_path / "bad")
    open(bad, "wb").write(bytes(data))
    same = ctx.integral(_spec(cg.FP64))
    with pytest.raises(cg.CubaGpuError, match="Sobol index"):
        same.load(bad)
    same.load(path)
    same.step(1)
    assert same.result().iterations == 3
    same.close()
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
