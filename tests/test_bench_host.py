"""Host logic of bench.py (CPU): the algorithmic FLOP count behind the
roofline, the peak formula, the sigma distance, the summary of the legs
and the lookup of committed profile figures by kernel source hash."""
import math
import os
import re

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_flops_per_sample_of_the_headline_workload():
    # genz8d4c: map 3 x 8, histogram 8 + 1, per component 10 for the sums,
    # and the families' own: oscillatory 2 x 8 + 2, product peak 4 x 8,
    # corner peak 2 x 8 + 4 (x^9 by squaring: 3 squarings, 1 multiply),
    # Gaussian 4 x 8 + 1
    assert bench.alg_flops_per_sample(8, [0, 1, 2, 3]) == 24 + 9 + 4 * 10 + 18 + 32 + 20 + 33 == 176


@pytest.mark.parametrize("ndim", [1, 3, 17, 32])
def test_flops_per_sample_grow_by_family_and_dimension(ndim):
    base = 3 * ndim + ndim + 1
    assert bench.alg_flops_per_sample(ndim, [6]) == base + 10  # the constant: the sums only
    assert bench.alg_flops_per_sample(ndim, [3]) == base + 10 + 4 * ndim + 1
    assert bench.alg_flops_per_sample(ndim, [3, 3]) == base + 2 * (10 + 4 * ndim + 1)


@pytest.mark.parametrize("e,muls", [(1, 0), (2, 1), (3, 2), (9, 4), (16, 4), (33, 6)])
def test_power_by_squaring_count(e, muls):
    # squarings up to the top bit, one multiply per further set bit
    assert bench._ipow_muls(e) == muls
    assert muls == (e.bit_length() - 1) + (bin(e).count("1") - 1)


def test_fp32_peak():
    assert bench.fp32_peak_tflops(2070.0, 152) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


def test_sigma_distance():
    assert bench._z(1.1, 0.05, 1.0) == pytest.approx(2.0)
    assert bench._z(1.0, 0.0, 1.0) == 0.0
    assert math.isinf(bench._z(1.5, 0.0, 1.0))


def test_max_over_ranks_without_a_process_group():
    assert bench.max_over_ranks(3.5) == 3.5


def _line(issue=True):
    line = {"value": 1.07e11, "e2e": {"value": 1.05e11},
            "roofline": {"frac": 0.2549, "kernel_ms": 0.0857, "issue": {"frac": 0.7} if issue else None},
            "plain_fp64": {"value": 1.88e9},
            "batch4096": {"value": 1.258e11, "plain_fp64_subset": {"value": 4.26e9},
                          "roofline": {"frac": 0.113, "issue": {"frac": 0.66} if issue else None}},
            "materialised": {"value": 4.53e10, "hbm_frac_all_kernels": 0.64},
            "accuracy": {"headline": {"z": [0.0066, 0.00075, 0.74, 0.00071]},
                         "batch4096": {"z_max": 28.0, "within_3": 0.9917,
                                       "oracle_subset": {"max_diff_in_sigma": 0.0059}}}}
    return line


@pytest.mark.parametrize("issue", [True, False])
def test_legs_summary(issue):
    out = bench.legs_summary(_line(issue))
    h = out["headline"]
    assert h["Gsps"] == 107.0 and h["e2e_Gsps"] == 105.0 and h["frac"] == 0.255
    assert h["kernel_us"] == 85.7 and h["z"] == [0.0066, 0.00075, 0.74, 0.00071]
    assert h["issue_frac"] == (0.7 if issue else None)
    b = out["batch4096"]
    assert b["Gsps"] == 125.8 and b["issue_frac"] == (0.66 if issue else None)
    assert b["z_max"] == 28.0 and b["oracle_dz"] == 0.0059
    assert out["materialised"] == {"Gsps": 45.3, "hbm_frac": 0.64, "z": []}
    assert out["plain_fp64"]["Gsps"] == 1.88


def _sha(name):
    text = open(os.path.join(ROOT, "profiles", name)).read()
    m = re.search(r"- source_sha: `([0-9a-f]+)`", text)
    return m.group(1) if m else None


@pytest.mark.parametrize("name,key", [("sampling_specialised_genz8d4c.md", "traffic_bytes_per_launch"),
                                      ("k_batch_sample_batch4096.md", "warp_instructions_per_run")])
def test_profile_figures_only_for_the_current_sources(name, key):
    v = bench._profile_value(name, key)
    if _sha(name) == bench._kernel_source_hash():
        assert isinstance(v, float) and v > 0
    else:
        assert v is None
    assert bench._profile_value("no_such_profile.md", key) is None
    assert bench._profile_value(name, "no_such_key") is None
