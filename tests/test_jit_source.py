"""The run-time specialised sampling kernel compiles for representative
problems (NVRTC needs no GPU): power-of-two bins with warp-private
histograms, power-of-two bins with block histograms, other bin counts,
one and many dimensions, every Genz family, scrambled and pseudo-random
points."""
import numpy as np
import pytest

import paper_1408_6373_gb300 as cg

CASES = [
    (8, [cg.OSCILLATORY, cg.PRODUCT_PEAK, cg.CORNER_PEAK, cg.GAUSSIAN], 128, 0),
    (1, [cg.DISCONTINUOUS], 50, 0),
    (30, [cg.C0, cg.DISCONTINUOUS], 256, 0),
    (16, [cg.PRODUCT_PEAK], 64, 0),
    (3, [cg.GAUSSIAN, cg.C0, cg.OSCILLATORY], 16, 0),
    (8, [cg.OSCILLATORY, cg.GAUSSIAN], 128, cg.SCRAMBLE),
    (7, [cg.CORNER_PEAK], 64, cg.PSEUDO),
]


def test_specialised_source_with_delay_compiles():
    g = cg.genz(5, [cg.GAUSSIAN], 1.0, 0.5, delay=300)
    ok, why = cg.jit_check(g, 64)
    if not ok and "libnvrtc" in why:
        pytest.skip(why)
    assert ok, why


@pytest.fixture(scope="module", autouse=True)
def _built():
    cg.build_library()


@pytest.mark.parametrize("ndim,fams,nbins,flags", CASES)
def test_specialised_source_compiles(ndim, fams, nbins, flags):
    rng = np.random.default_rng(ndim)
    g = cg.genz(ndim, fams, 0.5 + rng.random((len(fams), ndim)), rng.random((len(fams), ndim)))
    ok, why = cg.jit_check(g, nbins, flags)
    if not ok and "libnvrtc" in why:
        pytest.skip(why)
    assert ok, why


def test_invalid_problem_is_refused():
    g = cg.genz(2, [cg.GAUSSIAN], 1.0, 0.5)
    with pytest.raises(cg.CubaGpuError):
        cg.jit_check(g, 1)
