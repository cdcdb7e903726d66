"""The large single-integral configuration at full size: ndim 30, 256
bins, 1e9 Sobol points per iteration, indices beyond 2^32 (64-bit index
arithmetic), in the launch configuration the library uses for it.  The
oracle cannot evaluate 1e9 points in a test, so full-size passes are
checked by properties that hold at any size (f = 1 gives exact sums and
exact per-bin counts), by sampled outputs the oracle computes one by one
(Sobol points at those indices), and by the Genz closed forms."""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def test_full_size_pass_exact_counts_beyond_2_32(ctx):
    # one 1e9-point pass (rounded to a multiple of 256 x 2^k) starting at
    # 14 * 2^30 (> 2^33): f = 1 on the uniform power-of-two grid gives
    # S1 = S2 = n and n/256 points in every bin of every axis.
    ndim, N = 30, 256
    n = 2 ** 30
    start = 14 * 2 ** 30
    g = cg.genz(ndim, [cg.CONST], 1.0, 0.5)
    e = torch.tensor(O.grid_uniform(ndim, N), device="cuda")
    S1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    S2 = torch.zeros_like(S1)
    H = torch.zeros((ndim, N), dtype=torch.float64, device="cuda")
    ctx.sample(g, N, e, start, n, 0, S1, S2, H)
    ctx.synchronize()
    assert S1.item() == n and S2.item() == n
    assert torch.all(H == n // N).item()


@pytest.mark.parametrize("bits", [23, 52])
def test_sampled_points_beyond_2_32_bit_exact(ctx, bits):
    ndim = 30
    for start in (2 ** 32 - 5, 14 * 10 ** 9 + 12345, 15 * 10 ** 9 - 100):
        Y = torch.empty((ndim, 300), dtype=torch.int64, device="cuda")
        ctx.sobol(ndim, start, 300, bits, Y)
        ctx.synchronize()
        assert np.array_equal(Y.cpu().numpy().view(np.uint64), O.sobol_coords(ndim, start, 300, bits))


def test_large30d_within_closed_form():
    # the full configuration: 15 iterations x 1e9 points, both integrals
    c = cg.Context(0)
    for p in W.large30d():
        g = cg.genz(p.ndim, p.families, p.a, p.u)
        r = c.vegas(g, flags=0, maxeval=p.maxeval, nstart=p.nstart, nbins=p.nbins)
        exact = O.genz_exact(p.families[0], p.a[0], p.u[0])
        assert r.neval == p.maxeval
        assert abs(r.integral[0] - exact) <= 3 * r.error[0] + 1e-6 * abs(exact), (p.families, r.integral, exact, r.error)
    c.close()
