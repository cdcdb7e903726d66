"""Seeded synthetic workloads (inputs only -- none of the method's arithmetic).

The paper times Cuba on the 11 integrands of its demo program with a
calibrated delay loop (Sect. 4.1); those integrands are not available here,
so the Genz (1984) test families stand in for them.  Parameters are drawn
with SplitMix64 (Steele, Lea and Flood 2014) so every machine generates the
same inputs: u = (z >> 11) 2^-53 for each 64-bit output z, drawn
component-major, a-values first.

Workloads (sizes as the benchmark configurations name them):
  gaussian3d   ndim 3, Gaussian a_i = 5, u_i = 1/2, 50 bins, 10 x 1e4, FP64
  genz8d4c     ndim 8, components (oscillatory, product peak, corner peak,
               Gaussian), a,u ~ U(0,1) with each component's a scaled to
               sum 8, 128 bins, 20 x 1e7, FP32 evaluation
  batch4096    4096 integrals, ndim ~ U{2..16}, family ~ U{0..5}, points per
               iteration log-uniform in [1e4, 1e7], 10 iterations, 64 bins
  serve        Poisson arrivals, ndim ~ U{2..32}, ncomp ~ U{1..4}, epsrel
               log-uniform in [1e-5, 1e-3], maxeval 1e8 (a corner-peak
               component's a scaled down where needed: fp32_corner_peak)
  large30d     ndim 30, C0 and discontinuous, a_i = 1/2, u ~ U(0,1),
               256 bins, 15 x 1e9
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea, Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next() >> 11) * 2.0 ** -53

    def uniforms(self, n: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(n)])

    def integer(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def log_uniform(self, lo: float, hi: float) -> float:
        return math.exp(math.log(lo) + self.uniform() * (math.log(hi) - math.log(lo)))


@dataclass
class Problem:
    """One integral's inputs."""
    ndim: int
    families: list
    a: np.ndarray            # [ncomp, ndim]
    u: np.ndarray            # [ncomp, ndim]
    nbins: int
    nstart: int
    nincrease: int
    maxeval: int
    epsrel: float = 0.0
    epsabs: float = 0.0
    fp64: bool = False
    meta: dict = field(default_factory=dict)

    @property
    def ncomp(self) -> int:
        return len(self.families)

    @property
    def iterations(self) -> int:
        return self.maxeval // self.nstart if self.nincrease == 0 else -1


def fp32_corner_peak(a: np.ndarray) -> np.ndarray:
    """A corner-peak component's parameters scaled (down only) so that its
    value at the cube's centre, (1 + sum a / 2)^-(ndim+1), is at least
    2^-48: its squares then stay well inside binary32's normal range, which
    the FP32 path's sums of (J f)^2 need (in high dimensions the unscaled
    U(1/2, 3/2) draws put the values near 2^-120 and their squares below
    2^-126)."""
    a = np.asarray(a, dtype=np.float64)
    ndim = a.shape[-1]
    smax = 2.0 * (2.0 ** (48.0 / (ndim + 1)) - 1.0)
    s = a.sum(axis=-1, keepdims=True)
    return a * np.minimum(1.0, smax / s)


def gaussian3d() -> Problem:
    return Problem(3, [3], np.full((1, 3), 5.0), np.full((1, 3), 0.5), nbins=50,
                   nstart=10 ** 4, nincrease=0, maxeval=10 * 10 ** 4, fp64=True)


def genz8d4c(seed: int = 1, n_per_iter: int = 10 ** 7, iters: int = 20) -> Problem:
    rng = SplitMix64(seed)
    ndim, fams = 8, [0, 1, 2, 3]
    a = np.zeros((4, ndim))
    u = np.zeros((4, ndim))
    for c in range(4):
        a[c] = rng.uniforms(ndim)
        u[c] = rng.uniforms(ndim)
        a[c] *= 8.0 / a[c].sum()
    return Problem(ndim, fams, a, u, nbins=128, nstart=n_per_iter, nincrease=0,
                   maxeval=iters * n_per_iter)


def batch4096(seed: int = 3, count: int = 4096, iters: int = 10,
              nmin: float = 1e4, nmax: float = 1e7) -> list:
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        ndim = rng.integer(2, 16)
        fam = rng.integer(0, 5)
        n = int(round(rng.log_uniform(nmin, nmax)))
        a = 0.5 + rng.uniforms(ndim)
        u = rng.uniforms(ndim)
        out.append(Problem(ndim, [fam], a[None, :], u[None, :], nbins=64, nstart=n,
                           nincrease=0, maxeval=iters * n))
    return out


def serve_requests(seed: int = 4, rate: float = 2000.0, duration: float = 10.0,
                   nstart: int = 10 ** 4, nincrease: int = 5 * 10 ** 4,
                   maxeval: int = 10 ** 8) -> list:
    """(arrival_time_s, Problem) pairs of a Poisson arrival stream."""
    rng = SplitMix64(seed)
    t, out = 0.0, []
    while True:
        t += -math.log(1.0 - rng.uniform()) / rate
        if t >= duration:
            break
        ndim = rng.integer(2, 32)
        ncomp = rng.integer(1, 4)
        fams = [rng.integer(0, 5) for _ in range(ncomp)]
        a = 0.5 + np.array([rng.uniforms(ndim) for _ in range(ncomp)])
        u = np.array([rng.uniforms(ndim) for _ in range(ncomp)])
        for c in range(ncomp):
            if fams[c] == 2:
                a[c] = fp32_corner_peak(a[c])
        eps = rng.log_uniform(1e-5, 1e-3)
        out.append((t, Problem(ndim, fams, a, u, nbins=64, nstart=nstart,
                               nincrease=nincrease, maxeval=maxeval, epsrel=eps)))
    return out


def large30d(seed: int = 5, n_per_iter: int = 10 ** 9, iters: int = 15) -> list:
    rng = SplitMix64(seed)
    ndim = 30
    out = []
    for fam in (4, 5):
        u = rng.uniforms(ndim)
        out.append(Problem(ndim, [fam], np.full((1, ndim), 0.5), u[None, :], nbins=256,
                           nstart=n_per_iter, nincrease=0, maxeval=iters * n_per_iter))
    return out
