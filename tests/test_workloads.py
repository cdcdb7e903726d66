"""The seeded input generators (host logic, no GPU): SplitMix64 as Steele,
Lea and Flood define it (a 64-bit Weyl sequence with increment
0x9E3779B97F4A7C15 through the variant-13 mixer), determinism per seed,
and every workload's shapes and value distributions as the benchmark
configurations state them."""
import math

import numpy as np

from paper_1408_6373_gb300 import workloads as W

M64 = (1 << 64) - 1


def _mix(z):
    # the finaliser as the SplitMix64 paper states it, written out again
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def test_splitmix64_is_mixed_weyl_sequence():
    for seed in (0, 1, 12345, M64):
        g = W.SplitMix64(seed)
        for k in range(1, 200):
            assert g.next() == _mix((seed + k * 0x9E3779B97F4A7C15) & M64)


def test_uniform_draws_are_53_bit_fractions_in_unit_interval():
    g = W.SplitMix64(7)
    x = np.array([g.uniform() for _ in range(20000)])
    assert x.min() >= 0.0 and x.max() < 1.0
    assert np.all(x * 2.0 ** 53 == np.floor(x * 2.0 ** 53))
    assert abs(x.mean() - 0.5) < 6 * math.sqrt(1 / 12 / x.size)
    counts = np.bincount((x * 20).astype(int), minlength=20)
    assert ((counts - 1000) ** 2 / 1000).sum() < 20 + 8 * math.sqrt(40)


def test_integer_and_log_uniform_ranges():
    g = W.SplitMix64(11)
    ints = [g.integer(2, 16) for _ in range(5000)]
    assert min(ints) == 2 and max(ints) == 16 and len(set(ints)) == 15
    logs = np.array([g.log_uniform(1e4, 1e7) for _ in range(5000)])
    assert logs.min() >= 1e4 and logs.max() <= 1e7
    assert abs(np.log10(logs).mean() - 5.5) < 0.05


def test_workloads_are_deterministic_per_seed():
    a, b = W.genz8d4c(), W.genz8d4c()
    assert np.array_equal(a.a, b.a) and np.array_equal(a.u, b.u)
    assert not np.array_equal(W.genz8d4c(seed=2).a, a.a)
    x, y = W.batch4096(count=50), W.batch4096(count=50)
    assert all(np.array_equal(p.a, q.a) and p.nstart == q.nstart for p, q in zip(x, y))


def test_gaussian3d_shape():
    p = W.gaussian3d()
    assert (p.ndim, p.families, p.nbins, p.nstart, p.iterations, p.fp64) == (3, [3], 50, 10 ** 4, 10, True)
    assert np.all(p.a == 5.0) and np.all(p.u == 0.5)


def test_genz8d4c_shape():
    p = W.genz8d4c()
    assert (p.ndim, p.families, p.nbins, p.nstart, p.iterations) == (8, [0, 1, 2, 3], 128, 10 ** 7, 20)
    np.testing.assert_allclose(p.a.sum(axis=1), 8.0, rtol=1e-14)
    assert np.all(p.a > 0) and np.all((p.u >= 0) & (p.u < 1))


def test_batch4096_shape_and_distributions():
    ps = W.batch4096()
    assert len(ps) == 4096
    nd = np.array([p.ndim for p in ps])
    fam = np.array([p.families[0] for p in ps])
    n = np.array([p.nstart for p in ps], dtype=float)
    assert nd.min() == 2 and nd.max() == 16 and len(set(nd)) == 15
    assert set(fam) == set(range(6)) and all(p.ncomp == 1 for p in ps)
    assert n.min() >= 1e4 and n.max() <= 1e7 and abs(np.log10(n).mean() - 5.5) < 0.05
    assert all(p.nbins == 64 and p.iterations == 10 and p.nincrease == 0 for p in ps)
    assert all(np.all((p.a >= 0.5) & (p.a < 1.5)) for p in ps)


def test_serve_stream_is_poisson_with_stated_mix():
    reqs = W.serve_requests(duration=10.0)
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] < 10.0
    assert abs(len(reqs) - 20000) < 5 * math.sqrt(20000)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 2000) < 5 * (1 / 2000) / math.sqrt(gaps.size)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05  # exponential gaps
    nd = np.array([r[1].ndim for r in reqs])
    nc = np.array([r[1].ncomp for r in reqs])
    eps = np.array([r[1].epsrel for r in reqs])
    assert nd.min() == 2 and nd.max() == 32 and nc.min() == 1 and nc.max() == 4
    assert eps.min() >= 1e-5 and eps.max() <= 1e-3 and abs(np.log10(eps).mean() + 4) < 0.05
    assert all(r[1].maxeval == 10 ** 8 and r[1].nbins == 64 for r in reqs)


def test_large30d_shape():
    ps = W.large30d()
    assert [p.families for p in ps] == [[4], [5]]
    for p in ps:
        assert (p.ndim, p.nbins, p.nstart, p.iterations) == (30, 256, 10 ** 9, 15)
        assert np.all(p.a == 0.5) and np.all((p.u >= 0) & (p.u < 1))
