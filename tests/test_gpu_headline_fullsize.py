"""The headline configuration at full size, in the launch configuration the
benchmark times: genz8d4c (ndim 8; oscillatory, product peak, corner peak,
Gaussian; 128 bins; 20 iterations x 1e7 Sobol points), FP32 with the
run-time specialised kernel, one device-resident integral.

- The run meets every component's Genz closed form within 3 sigma (plus
  1e-6 relative for the FP32 evaluation bias).
- One full 1e7-point pass over the run's final grid, sampled through the
  staged grid exactly as an iteration samples, against the oracle on the
  same grid, element by element, with the FP32 tolerances of
  tests/tolerances.py (S1 within 1e-6 of sum |J f|, S2 within 1e-6
  relative, the implied variance bound, the histogram within 1e-5 of its
  row maximum).
- f = 1 over an aligned full-size range gives exact sums and exactly n/N
  points in every bin of every axis.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from tests.tolerances import check_fp32_pass

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


@pytest.fixture(scope="module")
def run(ctx):
    p = W.genz8d4c()
    g = cg.genz(p.ndim, p.families, p.a, p.u)
    I = ctx.integral(cg.spec(g, nbins=p.nbins, flags=cg.JIT, maxeval=p.maxeval, nstart=p.nstart))
    I.reset()
    I.run()
    r = I.result()
    edges = I.grid()
    I.close()
    return p, g, r, edges


def test_headline_run_meets_closed_forms(run):
    p, _, r, _ = run
    assert r.neval == p.maxeval and r.iterations == 20
    for c, fam in enumerate(p.families):
        exact = O.genz_exact(fam, p.a[c], p.u[c])
        assert abs(r.integral[c] - exact) <= 3 * r.error[c] + 1e-6 * abs(exact), (c, r.integral[c], exact)


def test_full_size_pass_matches_oracle(ctx, run):
    p, g, _, edges = run
    n = p.nstart
    e = torch.tensor(edges, dtype=torch.float64, device="cuda")
    table = torch.empty((p.ndim, p.nbins, 2), dtype=torch.float32, device="cuda")
    ctx.stage_grid(p.ndim, p.nbins, cg.JIT, e, table)
    S1 = torch.zeros(4, dtype=torch.float64, device="cuda")
    S2, H = torch.zeros_like(S1), torch.zeros((p.ndim, p.nbins), dtype=torch.float64, device="cuda")
    ctx.sample_staged(g, p.nbins, table, 1, n, cg.JIT, S1, S2, H)
    ctx.synchronize()
    S1, S2, H = S1.cpu().numpy(), S2.cpu().numpy(), H.cpu().numpy()
    prob = O.Problem(p.ndim, list(p.families), p.a, p.u, nbins=p.nbins, bits=23)
    check_fp32_pass(S1, S2, H, O.sample_bounds(prob, edges, 1, n, nthreads=os.cpu_count() or 1), n)


def test_full_size_constant_gives_exact_counts(ctx):
    ndim, N = 8, 128
    n = (10 ** 7 // N) * N  # whole aligned blocks of N points: one point per bin in each
    g = cg.genz(ndim, [cg.CONST], 1.0, 0.5)
    edges = np.tile(np.arange(N + 1) / N, (ndim, 1))
    e = torch.tensor(edges, dtype=torch.float64, device="cuda")
    table = torch.empty((ndim, N, 2), dtype=torch.float32, device="cuda")
    ctx.stage_grid(ndim, N, cg.JIT, e, table)
    S1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    S2, H = torch.zeros_like(S1), torch.zeros((ndim, N), dtype=torch.float64, device="cuda")
    ctx.sample_staged(g, N, table, N, n, cg.JIT, S1, S2, H)
    ctx.synchronize()
    assert S1.item() == n and S2.item() == n
    assert np.array_equal(H.cpu().numpy(), np.full((ndim, N), n // N, dtype=np.float64))
