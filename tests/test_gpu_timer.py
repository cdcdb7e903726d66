"""cv_kernel_timer / cv_kernel_times: one event pair per sampling launch made
outside stream capture, none for an integral's captured iterations, and
nothing once the timer is stopped."""
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
    return cg.genz(5, [cg.GAUSSIAN, cg.C0], np.full((2, 5), 1.0), np.full((2, 5), 0.3))


def test_each_sampling_launch_is_timed(ctx):
    g = _problem()
    e = torch.tensor(np.tile(np.linspace(0, 1, 65), (5, 1)), dtype=torch.float64, device="cuda")
    S1 = torch.zeros(2, dtype=torch.float64, device="cuda")
    S2 = torch.zeros_like(S1)
    H = torch.zeros((5, 64), dtype=torch.float64, device="cuda")
    ctx.kernel_timer(True)
    for k in range(3):
        ctx.sample(g, 64, e, 1 + k * 10 ** 6, 10 ** 6, 0, S1, S2, H)
    ctx.kernel_timer(False)
    t = ctx.kernel_times()
    assert len(t) == 3 and all(0.0 < x < 1000.0 for x in t)
    ctx.sample(g, 64, e, 1, 10 ** 6, 0, S1, S2, H)  # stopped: not recorded
    assert ctx.kernel_times() == t
    ctx.kernel_timer(True)  # a new start clears the record
    assert ctx.kernel_times() == []
    ctx.kernel_timer(False)


def test_vegas_iterations_timed_captured_iterations_not(ctx):
    g = _problem()
    ctx.kernel_timer(True)
    r = ctx.vegas(g, maxeval=5 * 10 ** 4, nstart=10 ** 4, nincrease=0, nbins=64)
    n_vegas = len(ctx.kernel_times())
    assert n_vegas == r.neval // 10 ** 4 == 5
    sp = cg.spec(g, nbins=64, maxeval=5 * 10 ** 4, nstart=10 ** 4, nincrease=0)
    I = ctx.integral(sp)
    I.run()  # iterations replayed from a captured graph
    ctx.synchronize()
    assert len(ctx.kernel_times()) == n_vegas
    I.close()
    ctx.kernel_timer(False)


def test_record_stops_at_its_capacity(ctx):
    g = _problem()
    e = torch.tensor(np.tile(np.linspace(0, 1, 65), (5, 1)), dtype=torch.float64, device="cuda")
    S1 = torch.zeros(2, dtype=torch.float64, device="cuda")
    S2 = torch.zeros_like(S1)
    H = torch.zeros((5, 64), dtype=torch.float64, device="cuda")
    ctx.kernel_timer(True)
    for k in range(cg.KERNEL_TIMER_CAP + 5):
        ctx.sample(g, 64, e, 1 + 4096 * k, 4096, 0, S1, S2, H)
    ctx.kernel_timer(False)
    assert len(ctx.kernel_times()) == cg.KERNEL_TIMER_CAP
