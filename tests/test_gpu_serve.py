"""GPU tests of the serving loop (cv_server_*): continuous batching of
requests with different ndim, ncomp and goals; each result equals the same
request run alone; admission by the device-memory budget; statistics."""
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import paper_1408_6373_gb300 as cg  # noqa: E402
from paper_1408_6373_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cg.build_library()
    c = cg.Context(0)
    yield c
    c.close()


def _request(rng):
    ndim = int(rng.integers(2, 33))
    ncomp = int(rng.integers(1, 5))
    fams = [int(f) for f in rng.integers(0, 6, ncomp)]
    a = 0.5 + rng.random((ncomp, ndim))
    u = rng.random((ncomp, ndim))
    for c in range(ncomp):
        if fams[c] == cg.CORNER_PEAK:
            a[c] = W.fp32_corner_peak(a[c])
    eps = float(np.exp(rng.uniform(np.log(1e-4), np.log(1e-2))))
    g = cg.genz(ndim, fams, a, u)
    return cg.spec(g, nbins=64, epsrel=eps, maxeval=2 * 10 ** 6, nstart=4000, nincrease=8000)


def _close(r, ref, nc):
    assert (r.neval, r.fail, r.iterations) == (ref.neval, ref.fail, ref.iterations)
    for c in range(nc):
        assert abs(r.integral[c] - ref.integral[c]) <= 2e-5 * abs(ref.integral[c]) + 1e-2 * ref.error[c]


def test_each_result_same_alone_and_in_the_mix(ctx):
    # every request served in a mix of 40 equals the same request served
    # alone, bit for bit (its tiles do not depend on the mix and their
    # partial rows are added in tile order); and it agrees with cv_vegas
    # (which groups points differently) within the FP32 tolerance
    rng = np.random.default_rng(7)
    specs = [_request(rng) for _ in range(40)]
    S = ctx.server(hbm_budget_bytes=256 << 20)
    ids = [S.submit(sp) for sp in specs]
    res = [S.wait(i, 120000) for i in ids]
    st = S.stats()
    S.stop()
    assert st.completed == 40 and st.max_live > 1
    for k in (0, 7, 19, 39):
        sp, r = specs[k], res[k]
        A = ctx.server()
        alone = A.wait(A.submit(sp), 120000)
        A.stop()
        assert (r.neval, r.fail, r.iterations) == (alone.neval, alone.fail, alone.iterations)
        for c in range(sp.g.ncomp):
            for key in ("integral", "error", "prob"):
                x, y = getattr(r, key)[c], getattr(alone, key)[c]
                assert np.float64(x).view(np.uint64) == np.float64(y).view(np.uint64), (k, c, key, x, y)
    # against the mathematics: every served estimate within 3 sigma of its
    # Genz closed form, plus the mixed-precision bound 1e-6 int |f| (the FP32
    # evaluation's distance from the FP64 one on the same grid; it matters
    # where an oscillatory integral nearly cancels).  A miss is accepted only
    # where Vegas itself misses: the oracle's FP64 Vegas run of the same
    # request -- every component, the same points, schedule and goal (the
    # grid follows component 0, so a later component can be sampled badly
    # and its error underestimated) -- must then be more than 2 sigma off as
    # well, and both misses are listed in the message.
    misses, total, oracle_runs = [], 0, {}
    for k, (sp, r) in enumerate(zip(specs, res)):
        nd, nc = sp.g.ndim, sp.g.ncomp
        fams = [sp.g.family[c] for c in range(nc)]
        a = np.array([sp.g.a[c][:nd] for c in range(nc)])
        u = np.array([sp.g.u[c][:nd] for c in range(nc)])
        for c in range(nc):
            total += 1
            ex = O.genz_exact(fams[c], a[c], u[c])
            p1 = O.Problem(nd, [fams[c]], a[c][None], u[c][None], nbins=sp.nbins)
            absint = O.sample_bounds(p1, O.grid_uniform(nd, sp.nbins), 1, 1 << 14).A1[0] / (1 << 14)
            z = abs(r.integral[c] - ex) / max(3 * r.error[c] + 1e-6 * absint, 1e-300) * 3
            if z >= 3:
                if k not in oracle_runs:
                    p = O.Problem(nd, fams, a, u, nbins=sp.nbins)
                    oracle_runs[k] = O.vegas(p, epsrel=sp.epsrel, maxeval=sp.maxeval, nstart=sp.nstart,
                                             nincrease=sp.nincrease, nthreads=16)
                o = oracle_runs[k]
                zo = abs(o.integral[c] - ex) / max(o.error[c], 1e-300)
                misses.append((k, c, nd, fams[c], round(z, 2), round(zo, 2)))
    assert all(m[5] > 2 for m in misses), misses
    assert total > 60


def test_arrivals_while_busy_join_later_rounds(ctx):
    rng = np.random.default_rng(8)
    S = ctx.server(hbm_budget_bytes=64 << 20)
    first = [S.submit(_request(rng)) for _ in range(8)]
    time.sleep(0.002)
    late = [S.submit(_request(rng)) for _ in range(8)]
    out = [S.wait(i, 120000) for i in first + late]
    st = S.stats()
    S.stop()
    assert all(r.neval > 0 for r in out)
    assert st.rounds >= max(r.iterations for r in out)
    assert st.p50_ms > 0 and st.p99_ms >= st.p50_ms


def test_budget_admission_and_rejection(ctx):
    rng = np.random.default_rng(9)
    sp = _request(rng)
    # 20 dimensions x 256 bins need 82,688 bytes of state: a 120 KB budget
    # holds one such request at a time, and all still complete, one by one
    def big():
        g = cg.genz(20, [cg.GAUSSIAN], 0.5 + rng.random(20), rng.random(20))
        return cg.spec(g, nbins=256, maxeval=3 * 5000, nstart=5000)
    S = ctx.server(hbm_budget_bytes=120 * 1024)
    ids = [S.submit(big()) for _ in range(5)]
    res = [S.wait(i, 120000) for i in ids]
    st = S.stats()
    assert st.max_live == 1 and all(r.neval > 0 for r in res)
    # a request that can never fit is refused at submission
    tiny = ctx.server(hbm_budget_bytes=4096)
    with pytest.raises(cg.CubaGpuError) as ei:
        tiny.submit(sp)
    assert ei.value.code == cg.EADMIT
    tiny.stop()
    # too many bins for the batched kernel's shared memory: refused
    wide = cg.spec(cg.genz(32, [cg.GAUSSIAN], 1.0, 0.5), nbins=256, maxeval=10000, nstart=5000)
    with pytest.raises(cg.CubaGpuError) as ei:
        S.submit(wide)
    assert ei.value.code == cg.EINVAL
    S.stop()


def test_submit_from_two_threads_and_poll(ctx):
    rng = np.random.default_rng(10)
    specs = [_request(rng) for _ in range(16)]
    S = ctx.server()
    ids = [None] * 16

    def worker(k0):
        for k in range(k0, 16, 2):
            ids[k] = S.submit(specs[k])

    th = [threading.Thread(target=worker, args=(k,)) for k in (0, 1)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert len(set(ids)) == 16
    deadline = time.time() + 120
    pending = set(ids)
    while pending and time.time() < deadline:
        pending = {i for i in pending if S.poll(i) is None}
        time.sleep(0.001)
    assert not pending
    with pytest.raises(cg.CubaGpuError) as ei:
        S.poll(10 ** 9)
    assert ei.value.code == cg.ENOTFOUND
    S.stop()


def test_stop_finishes_submitted_requests(ctx):
    rng = np.random.default_rng(11)
    S = ctx.server()
    ids = [S.submit(_request(rng)) for _ in range(6)]
    st_before = S.stats()
    S.stop()  # waits for every submitted request
    assert st_before.submitted == 6
