"""FP32 sampling passes of 9 to 32 dimensions against the FP64 oracle,
element by element, on the same seeded inputs and grid.

These dimensions run their own kernel instantiations: the two-CTA-per-SM,
128-register build for 9-32 dimensions, the 256-bin bit-permuted direction
table, and the run-time specialised kernel (CV_JIT) that the large
30-dimensional integral and the 17-32-dimensional serving classes use.  The
cases reach Sobol indices past 2^32 and passes of a million points (several
thousand 32-point blocks per warp chunk), with ragged ends.  Tolerances are
the FP32 ones of tests/tolerances.py (1e-6 of sum |J f| plus the boundary
mass for S1, 1e-6 relative plus boundary mass for S2, the implied variance
bound, the histogram within 1e-5 of its row maximum)."""
import os

import numpy as np
import pytest

import oracle as O
from tests.tolerances import check_fp32_pass

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1408_6373_gb300 as cg  # noqa: E402
from paper_1408_6373_gb300 import workloads as W  # noqa: E402

THREADS = os.cpu_count() or 1

# (ndim, nbins, families, start, n)
CASES = [
    (9, 64, [O.GAUSSIAN, O.OSCILLATORY, O.PRODUCT_PEAK, O.CORNER_PEAK], 1, 200001),
    (9, 256, [O.C0, O.DISCONTINUOUS], 77, 300000),
    (16, 64, [O.CORNER_PEAK, O.GAUSSIAN], 2 ** 33 + 5, 2 ** 20),
    (16, 256, [O.OSCILLATORY, O.C0, O.DISCONTINUOUS], 12345, 250003),
    (17, 64, [O.PRODUCT_PEAK, O.GAUSSIAN, O.OSCILLATORY], 3, 300001),
    (17, 256, [O.DISCONTINUOUS], 2 ** 32 - 1000, 200000),
    (24, 64, [O.GAUSSIAN, O.C0], 1, 150001),
    (24, 256, [O.OSCILLATORY, O.DISCONTINUOUS], 2 ** 34 + 31, 150000),
    (30, 64, [O.C0, O.DISCONTINUOUS], 1, 120001),
    (30, 256, [O.C0, O.DISCONTINUOUS], 2 ** 32 + 12345, 1000003),
    (32, 64, [O.PRODUCT_PEAK, O.GAUSSIAN, O.OSCILLATORY, O.C0], 99, 100000),
    (32, 256, [O.DISCONTINUOUS, O.GAUSSIAN], 2 ** 33, 100001),
]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cg.build_library()
    c = cg.Context(0)
    yield c
    c.close()


def _inputs(case):
    ndim, nbins, fams, start, n = case
    rng = np.random.default_rng(1000 * ndim + nbins)
    a = rng.uniform(0.5, 1.5, (len(fams), ndim))
    u = rng.uniform(0.1, 0.9, (len(fams), ndim))
    for c, f in enumerate(fams):
        if f in (O.C0, O.DISCONTINUOUS):
            a[c] = 0.5  # the large single integral's parameters
        elif f == O.CORNER_PEAK:
            a[c] = W.fp32_corner_peak(a[c])  # inside the FP32 path's range
    w = rng.uniform(0.2, 1.0, (ndim, nbins))
    cs = np.concatenate([np.zeros((ndim, 1)), np.cumsum(w, axis=1)], axis=1)
    edges = cs / cs[:, -1:]
    edges[:, 0], edges[:, -1] = 0.0, 1.0
    return a, u, edges


_oracle_cache = {}


def _oracle(case):
    if case[:2] not in _oracle_cache:
        ndim, nbins, fams, start, n = case
        a, u, edges = _inputs(case)
        p = O.Problem(ndim, fams, a, u, nbins=nbins, bits=23)
        _oracle_cache[case[:2]] = O.sample_bounds(p, edges, start, n, nthreads=THREADS)
    return _oracle_cache[case[:2]]


@pytest.mark.parametrize("flags", [0, cg.JIT], ids=["generic", "jit"])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}d-{c[1]}bins" for c in CASES])
def test_fp32_pass_high_dimensions(ctx, case, flags):
    ndim, nbins, fams, start, n = case
    a, u, edges = _inputs(case)
    g = cg.genz(ndim, fams, a, u)
    e = torch.tensor(edges, dtype=torch.float64, device="cuda")
    S1 = torch.zeros(len(fams), dtype=torch.float64, device="cuda")
    S2 = torch.zeros_like(S1)
    H = torch.zeros((ndim, nbins), dtype=torch.float64, device="cuda")
    ctx.sample(g, nbins, e, start, n, flags, S1, S2, H)
    ctx.synchronize()
    S1, S2, H = (t.cpu().numpy() for t in (S1, S2, H))
    ob = _oracle(case)
    check_fp32_pass(S1, S2, H, ob, n, what=(ndim, nbins, flags))
    # the points reach the same bins (integer map on both sides)
    assert np.array_equal(H == 0, ob.H == 0)


@pytest.mark.parametrize("case", [CASES[3], CASES[9]], ids=["16d-256bins", "30d-256bins"])
def test_fp32_staged_pass_high_dimensions(ctx, case):
    # the pass as an integral's iteration runs it: the grid staged once into
    # the FP32 table and the specialised kernel reading it
    ndim, nbins, fams, start, n = case
    a, u, edges = _inputs(case)
    g = cg.genz(ndim, fams, a, u)
    e = torch.tensor(edges, dtype=torch.float64, device="cuda")
    table = torch.empty((ndim, nbins, 2), dtype=torch.float32, device="cuda")
    ctx.stage_grid(ndim, nbins, cg.JIT, e, table)
    S1 = torch.zeros(len(fams), dtype=torch.float64, device="cuda")
    S2 = torch.zeros_like(S1)
    H = torch.zeros((ndim, nbins), dtype=torch.float64, device="cuda")
    ctx.sample_staged(g, nbins, table, start, n, cg.JIT, S1, S2, H)
    ctx.synchronize()
    check_fp32_pass(*(t.cpu().numpy() for t in (S1, S2, H)), _oracle(case), n, what="staged")
