#!/usr/bin/env python3
"""Benchmark of the GB300 Vegas sampling path.

One step = one complete Vegas integration of the mixed-precision Genz
workload (ndim 8, four components: oscillatory, product peak, corner peak,
Gaussian; 20 iterations x 1e7 Sobol points; 128 bins per axis): reset of
the device-resident grid and sums, then every iteration's fused sampling
pass, FP64 refinement and FP64 combination, replayed from a CUDA graph.

Printed (one JSON line on rank 0):
  value      samples/s over all ranks, device-timed with CUDA events, inputs
             resident, L2 flushed (256 MiB write) before every step
  e2e        samples/s through the public call cv_vegas (host integrand
             description in, host results out) timed on the host
  roofline   the fused sampling kernel against the FP32 pipe peak
             (152 SMs x 128 lanes x 2 flop x the maximum SM clock)
  cpu_baseline  the FP64 CPU oracle on the host cores, bounded sample
  plain_fp64 the FP64 one-launch-per-iteration comparator, same workload

--impl reference times the CPU oracle instead (the reference arm).
Multi-GPU (torchrun): every rank runs its own replica of the workload
(weak scaling); the slowest rank's time is reported.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Vegas samples/s"
UNIT = "samples/s"
FP32_LANES_PER_SM = 128


def sm_count(device: int = 0) -> int:
    """Streaming multiprocessors of the device, queried at run time."""
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def _workload_name(p) -> str:
    return (f"genz8d4c: Vegas FP32 eval / FP64 reduce, ndim {p.ndim}, ncomp {p.ncomp} "
            f"(oscillatory, product peak, corner peak, gaussian), {p.maxeval // p.nstart} iterations "
            f"x {p.nstart:.0e} Sobol points, {p.nbins} bins")


# ------------------------------------------------------------------ FLOP count
def alg_flops_per_sample(ndim: int, families) -> int:
    """Algorithmic FP32 FLOPs of one sample of the fused pass (FMA = 2; the
    special-function unit's exp/cos/rcp are not FP32-pipe FLOPs): the map
    3/dim (the point's FMA and the Jacobian's multiply); per component J*f,
    (J f)^2 and two Kahan additions (4 each) = 10; the histogram, f0^2 and
    one addition per axis = ndim + 1; and the family's own arithmetic.  The
    count is of the method's work, not of the instructions a kernel issues
    (the FP32 kernel adds Newton steps and compensation terms for accuracy,
    which count against it)."""
    per = {
        0: 2 * ndim + 2,                      # phase FMAs, wrap, scale
        1: 4 * ndim,                          # sub, FMA, mul per dim
        2: 2 * ndim + _ipow_muls(ndim + 1),   # FMAs, power by squaring
        3: 4 * ndim + 1,                      # 2 FMA per dim, scale
        4: 3 * ndim + 1,                      # sub, FMA per dim, negate
        5: 2 * ndim + 1,
        6: 0,
    }
    return 3 * ndim + sum(per[f] + 10 for f in families) + ndim + 1


def _ipow_muls(e: int) -> int:
    return max(0, e.bit_length() - 1) + max(0, bin(e).count("1") - 1)


def fp32_peak_tflops(sm_mhz: float, sms: int) -> float:
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clock / throttle sampling every 20 ms, started before the
    timed region; only the samples taken inside the region (host clock,
    between mark_start and mark_end) are reported, or, if the region was
    shorter than the sampling period, the one sample nearest to it."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "20"]
        uuid = _gpu_uuid(device_index)
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        self.t0 = self.t1 = None
        time.sleep(0.3)  # (the sampler's first rows)

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()
        time.sleep(0.05)

    def stop(self) -> dict:
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        samples = []
        for r in rows:
            try:
                ts = time.mktime(time.strptime(r[0].strip().split(".")[0], "%Y/%m/%d %H:%M:%S"))
                ts += float("0." + r[0].strip().split(".")[1]) if "." in r[0] else 0.0
                samples.append((ts, float(r[1]), float(r[2]),
                                {nm for nm, v in zip(names, r[4:8]) if v.strip().lower() == "active"}))
            except (ValueError, IndexError):
                continue
        inside = [s for s in samples if self.t0 is not None and self.t0 <= s[0] <= (self.t1 or s[0])]
        basis = "inside the timed region"
        if not inside and samples and self.t0 is not None:
            mid = 0.5 * (self.t0 + (self.t1 or self.t0))
            inside = [min(samples, key=lambda s: abs(s[0] - mid))]
            basis = "nearest sample to a timed region shorter than the 20 ms period"
        reasons = set()
        for s in inside:
            reasons |= s[3]
        return {"sm_mhz": statistics.median(s[1] for s in inside) if inside else None,
                "sm_max_mhz": max(s[2] for s in inside) if inside else None,
                "reasons": sorted(reasons), "samples": len(inside), "period_ms": 20, "basis": basis}


class NvmlClockSampler:
    """The same record as ClockSampler, read through NVML (libnvidia-ml,
    loaded with ctypes) every 2 ms by a host thread: the SM clock, its
    maximum and the active clock-event reasons (NVML's bit mask).  Only
    reads: no setting of the GPU is touched."""
    PERIOD_S = 0.002
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device_index: int):
        import ctypes
        import threading
        uuid = _gpu_uuid(device_index)
        if not uuid:
            raise OSError("no device UUID")
        self.nv = ctypes.CDLL("libnvidia-ml.so.1")
        if self.nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        if self.nv.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) != 0:
            raise OSError("no NVML handle for " + uuid)
        self.ct = ctypes
        self.nv.nvmlDeviceGetCurrentClocksEventReasons  # (AttributeError on an older NVML)
        if self._read() is None:
            raise OSError("NVML clock queries failed")
        self.samples = []
        self.t0 = self.t1 = None
        self.run = True
        self.th = threading.Thread(target=self._loop, daemon=True)
        self.th.start()
        time.sleep(0.05)

    def _read(self):
        ct = self.ct
        mhz, mx, rs = ct.c_uint(), ct.c_uint(), ct.c_ulonglong()
        ok = (self.nv.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(mhz)) == 0 and
              self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ct.byref(mx)) == 0 and
              self.nv.nvmlDeviceGetCurrentClocksEventReasons(self.h, ct.byref(rs)) == 0)
        return (time.time(), float(mhz.value), float(mx.value),
                {nm for bit, nm in self.REASONS.items() if rs.value & bit}) if ok else None

    def _loop(self):
        while self.run:
            r = self._read()
            if r is not None:
                self.samples.append(r)
            time.sleep(self.PERIOD_S)

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()
        time.sleep(0.01)

    def stop(self) -> dict:
        self.run = False
        self.th.join(timeout=2)
        self.nv.nvmlShutdown()
        inside = [x for x in self.samples if self.t0 is not None and self.t0 <= x[0] <= (self.t1 or x[0])]
        basis = "NVML every 2 ms, samples inside the timed region"
        if not inside and self.samples and self.t0 is not None:
            mid = 0.5 * (self.t0 + (self.t1 or self.t0))
            inside = [min(self.samples, key=lambda x: abs(x[0] - mid))]
            basis = "NVML every 2 ms, nearest sample to the timed region"
        reasons = set()
        for x in inside:
            reasons |= x[3]
        return {"sm_mhz": statistics.median(x[1] for x in inside) if inside else None,
                "sm_max_mhz": max(x[2] for x in inside) if inside else None,
                "reasons": sorted(reasons), "samples": len(inside), "period_ms": 1e3 * self.PERIOD_S,
                "basis": basis}


def clock_sampler(device_index: int):
    """NVML sampling where the driver library loads, else nvidia-smi."""
    try:
        return NvmlClockSampler(device_index)
    except (OSError, AttributeError):
        return ClockSampler(device_index)


def _gpu_uuid(idx: int):
    try:
        import torch
        u = torch.cuda.get_device_properties(idx).uuid
        return f"GPU-{u}" if u else None
    except Exception:
        return None


# ------------------------------------------------------------------ helpers
def max_over_ranks(x: float, device=None) -> float:
    """The largest value of x over all ranks (the slowest rank's time); the
    value itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


KERNEL_SOURCES = ("cv_device.cuh", "cv_internal.cuh", "sobol_dirs.h", "cv_jit.cu")


def _kernel_source_hash() -> str:
    """Hash of the files that define the sampling kernel."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1408_6373_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _profile_traffic(name: str):
    """DRAM bytes per launch of the sampling kernel from the committed ncu
    summary `name`, if it was taken on the current kernel sources."""
    return _profile_value(name, "traffic_bytes_per_launch")


def _profile_value(name: str, key: str):
    """A figure ("- key: value") of the committed ncu summary `name`, if it
    was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, _, v = line.strip()[2:].partition(":")
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha") != _kernel_source_hash():
        return None
    try:
        return float(vals[key].split()[0])
    except (KeyError, ValueError, IndexError):
        return None


# ------------------------------------------------------------------ CPU oracle
def cpu_oracle_rate(p, target_s: float, threads: int):
    """Time the FP64 CPU oracle on a bounded sample of workload p: two
    iterations of n points, n sized for about target_s seconds."""
    import numpy as np

    import oracle as O
    prob = O.Problem(p.ndim, list(p.families), np.asarray(p.a), np.asarray(p.u),
                     nbins=p.nbins, bits=23)
    prob.directions()
    n0 = 2000 * threads
    t = time.perf_counter()
    O.vegas(prob, maxeval=n0, nstart=n0, nthreads=threads)
    rate0 = n0 / max(time.perf_counter() - t, 1e-6)
    n = max(n0, int(rate0 * target_s / 2))
    t = time.perf_counter()
    O.vegas(prob, maxeval=2 * n, nstart=n, nthreads=threads)
    dt = time.perf_counter() - t
    return 2 * n / dt, dt, n


def oracle_pass_rate(problems, cap: int, threads: int) -> tuple:
    """The oracle's sampling rate over a list of problems: one pass of
    min(nstart, cap) points each on the uniform grid (a Vegas iteration's
    sampling, its refinement left out), FP32-decided like the GPU path."""
    import numpy as np

    import oracle as O
    total, dt = 0, 0.0
    for p in problems:
        prob = O.Problem(p.ndim, list(p.families), np.asarray(p.a), np.asarray(p.u),
                         nbins=p.nbins, bits=23)
        prob.directions()
        e = O.grid_uniform(p.ndim, p.nbins)
        n = min(int(p.nstart), cap)
        t = time.perf_counter()
        O.sample(prob, e, 1, n, nthreads=threads)
        dt += time.perf_counter() - t
        total += n
    return total / dt, total, dt


def oracle_more_rates(p, W, threads: int) -> dict:
    """Further oracle figures of the CPU-baseline leg: the headline on one
    thread, and bounded samples of the batched and large workloads."""
    out = {}
    rate, dt, n = cpu_oracle_rate(p, 3.0, 1)
    out["single_thread"] = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"2 Vegas iterations x {n} points of the headline workload, {dt:.1f} s"}
    rate, total, dt = oracle_pass_rate(W.batch4096()[:64], 10 ** 6, threads)
    out["batch4096"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                        "sample": f"the first 64 of the 4096 integrals, one pass of min(n, 1e6) points each "
                                  f"({total} points, {dt:.1f} s)"}
    rate, total, dt = oracle_pass_rate(W.large30d(), 10 ** 8, threads)
    out["large30d"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                       "sample": f"both integrals, one pass of 1e8 points each (one of the 15 iterations the "
                                 f"oracle's share of the workload takes; {total} points, {dt:.1f} s)"}
    return out


def _z(I: float, E: float, exact: float) -> float:
    """Distance of an estimate from the exact value in units of its error."""
    if E > 0:
        return abs(I - exact) / E
    return 0.0 if I == exact else float("inf")


def accuracy_leg(line: dict, W, threads: int) -> dict:
    """Every result's distance from its Genz closed form in units of its own
    error estimate, z = |I - exact| / error, per leg (max and share within
    3), and the largest difference from the oracle's own Vegas run of the
    same integrals on seeded subsets.  Part of the CPU-baseline leg: the
    closed forms and the runs are the oracle's."""
    import numpy as np

    import oracle as O
    out = {}
    p = W.genz8d4c()
    ex = [O.genz_exact(f, np.asarray(p.a[c]), np.asarray(p.u[c])) for c, f in enumerate(p.families)]
    r = line["result"]
    out["headline"] = {"z": [_z(r["integral"][c], r["error"][c], ex[c]) for c in range(p.ncomp)]}
    out["plain_fp64"] = {"z": [_z(r["plain_fp64_integral"][c], r["plain_fp64_error"][c], ex[c])
                               for c in range(p.ncomp)]}
    if "materialised" in line:
        res = line["materialised"].pop("_results")
        out["materialised"] = {"z": [_z(I, E, ex[c]) for c, (I, E) in enumerate(res)]}
    if "generators" in line:
        gen = line["generators"]
        out["generators"] = {k: {"z": [_z(gen[k]["integral_mean"][c], gen[k]["vegas_error"][c], ex[c])
                                       for c in range(p.ncomp)]} for k in ("scrambled", "pseudo") if k in gen}
    if "gaussian3d" in line:
        g3 = line["gaussian3d"]
        out["gaussian3d"] = {"z": _z(g3["integral"], g3["error"], g3["exact"])}
    if "suave" in line:
        sv = line["suave"]
        P = SUAVE_PROBLEM
        exs = O.genz_exact(3, np.array(P["a"]), np.array(P["u"]))
        out["suave"] = {"z": _z(sv["integral"], sv["error"], exs)}
    if "large30d" in line:
        zl = []
        for item in line["large30d"]["results"]:
            q = item.pop("_p")
            zl.append(_z(item["integral"], item["error"], O.genz_exact(q.families[0], q.a[0], q.u[0])))
        out["large30d"] = {"z": zl}
    if "batch4096" in line:
        b = line["batch4096"]
        probs, res = b.pop("_problems"), b.pop("_results")
        exact = [O.genz_exact(q.families[0], q.a[0], q.u[0]) for q in probs]
        zs = np.array([_z(I, E, x) for (I, E), x in zip(res, exact)])
        plain = b["plain_fp64_subset"].pop("_results")
        zp = [_z(I, E, exact[i]) for i, (I, E) in plain]
        # the oracle's own Vegas run of the 8 integrals with the fewest points
        idx = sorted(range(len(probs)), key=lambda i: probs[i].maxeval)[:8]
        dz = []
        for i in idx:
            q = probs[i]
            o = O.vegas(O.Problem(q.ndim, list(q.families), np.asarray(q.a), np.asarray(q.u), nbins=q.nbins,
                                  bits=23), maxeval=q.maxeval, nstart=q.nstart, nthreads=threads)
            dz.append(abs(res[i][0] - o.integral[0]) / max(res[i][1], o.error[0]))
        out["batch4096"] = {"integrals": len(zs), "z_max": float(zs.max()), "within_3": float((zs <= 3).mean()),
                            "plain_fp64_subset_z_max": max(zp),
                            "oracle_subset": {"integrals": len(idx), "max_diff_in_sigma": max(dz)}}
    if "serve" in line:
        raw = line["serve"].pop("_results")
        zs, z0, zero_err, small = [], [], 0, []
        for q, rc, neval in raw:
            for c, (I, E) in enumerate(rc):
                x = O.genz_exact(q.families[c], np.asarray(q.a[c]), np.asarray(q.u[c]))
                # the mixed-precision bound 1e-6 int |f| (|f| <= 1 for the oscillatory family)
                floor = 1e-6 * (1.0 if q.families[c] == 0 else abs(x))
                if E == 0.0:
                    # (every sample of the component was zero, or constant:
                    # Vegas's 0 +- 0; counted, not given a z)
                    zero_err += 1
                    continue
                z = abs(I - x) / (E + floor / 3)
                zs.append(z)
                if c == 0:
                    z0.append(z)
            if len(small) < 5 and neval <= 3 * 10 ** 5:
                small.append((q, rc))
        zs, z0 = np.array(zs), np.array(z0)
        dz = []
        for q, rc in small:
            # the same request, goal and schedule (it stops where the GPU run stopped)
            o = O.vegas(O.Problem(q.ndim, list(q.families), np.asarray(q.a), np.asarray(q.u), nbins=q.nbins, bits=23),
                        epsrel=q.epsrel, maxeval=q.maxeval, nstart=q.nstart, nincrease=q.nincrease,
                        nthreads=threads)
            dz.append(max(abs(I - o.integral[c]) / max(E, o.error[c]) for c, (I, E) in enumerate(rc)))
        out["serve"] = {"components": len(zs), "z_max": float(zs.max()), "within_3": float((zs <= 3).mean()),
                        "component0": {"z_max": float(z0.max()), "within_3": float((z0 <= 3).mean()),
                                       "basis": "the component whose histogram refines the grid"},
                        "zero_error_components": int(zero_err),
                        "zero_error_basis": "components whose Vegas error is 0 (all samples zero or equal), left out of z",
                        "basis": "z with the FP32 floor 1e-6 int|f| added to 3 sigma; the grid follows component 0, "
                                 "so later components of a request can be sampled badly and their error "
                                 "underestimated by Vegas itself",
                        "oracle_subset": {"requests": len(dz), "max_diff_in_sigma": max(dz) if dz else None,
                                          "basis": "the first requests the GPU finished within 3e5 points, "
                                                   "rerun by the oracle with the same goal and schedule"}}
    return out


def legs_summary(line: dict) -> dict:
    """A short form of every leg, printed last on the line (so that a record
    that keeps only the end of the output still holds every leg)."""
    def g(v, nd=4):
        return float(f"{v:.{nd}g}") if isinstance(v, (int, float)) and v is not None else v
    acc = line.get("accuracy", {})
    iss = line["roofline"].get("issue") or {}
    out = {"headline": {"Gsps": g(line["value"] / 1e9), "e2e_Gsps": g(line["e2e"]["value"] / 1e9),
                        "frac": g(line["roofline"]["frac"], 3), "issue_frac": g(iss.get("frac"), 3),
                        "kernel_us": g(1e3 * line["roofline"]["kernel_ms"]),
                        "z": [g(z, 2) for z in acc.get("headline", {}).get("z", [])]},
           "plain_fp64": {"Gsps": g(line["plain_fp64"]["value"] / 1e9),
                          "z": [g(z, 2) for z in acc.get("plain_fp64", {}).get("z", [])]}}
    if "batch4096" in line:
        b, a = line["batch4096"], acc.get("batch4096", {})
        bi = b["roofline"].get("issue") or {}
        out["batch4096"] = {"Gsps": g(b["value"] / 1e9), "frac": g(b["roofline"]["frac"], 3),
                            "issue_frac": g(bi.get("frac"), 3),
                            "plain_fp64_Gsps": g(b["plain_fp64_subset"]["value"] / 1e9),
                            "z_max": g(a.get("z_max"), 3), "within_3": g(a.get("within_3"), 4),
                            "oracle_dz": g(a.get("oracle_subset", {}).get("max_diff_in_sigma"), 2)}
    if "large30d" in line:
        out["large30d"] = {"Gsps": g(line["large30d"]["value"] / 1e9),
                           "z": [g(z, 2) for z in acc.get("large30d", {}).get("z", [])]}
    if "materialised" in line:
        m = line["materialised"]
        out["materialised"] = {"Gsps": g(m["value"] / 1e9), "hbm_frac": g(m["hbm_frac_all_kernels"], 3),
                               "z": [g(z, 2) for z in acc.get("materialised", {}).get("z", [])]}
    if "serve" in line:
        s, a = line["serve"], acc.get("serve", {})
        out["serve"] = {"req_s": g(s["requests_per_s"]), "p50_ms": g(s["p50_ms"]), "p99_ms": g(s["p99_ms"]),
                        "Gsps": g(s["throughput"]["value"] / 1e9), "fifo_fp64_p50_ms": g(s["plain_fp64_fifo"]["p50_ms"]),
                        "z_max": g(a.get("z_max"), 3), "within_3": g(a.get("within_3"), 4),
                        "c0_within_3": g(a.get("component0", {}).get("within_3"), 4),
                        "oracle_dz": g(a.get("oracle_subset", {}).get("max_diff_in_sigma"), 2)}
    if "gaussian3d" in line:
        out["gaussian3d"] = {"us_it": g(line["gaussian3d"]["graph_us_per_iteration"]),
                             "z": g(acc.get("gaussian3d", {}).get("z"), 2)}
    if "suave" in line:
        out["suave"] = {"Gsps": g(line["suave"]["value"] / 1e9), "z": g(acc.get("suave", {}).get("z"), 2)}
    if "cpu_baseline" in line:
        out["oracle_Msps"] = g(line["cpu_baseline"]["value"] / 1e6)
    return out


def _strip_private(d):
    """Drop the raw results kept for the accuracy leg (keys starting with _)."""
    if isinstance(d, dict):
        return {k: _strip_private(v) for k, v in d.items() if not k.startswith("_")}
    if isinstance(d, list):
        return [_strip_private(v) for v in d]
    return d


# ------------------------------------------------------------------ arms
def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_1408_6373_gb300 import workloads as W
    p = W.genz8d4c()
    threads = os.cpu_count() or 1
    per_step_s = 3.0
    rates = []
    for i in range(args.warmup + args.steps):
        r, dt, n = cpu_oracle_rate(p, per_step_s, threads)
        if i >= args.warmup:
            rates.append((r, dt, n))
    tot_n = sum(2 * n for _, _, n in rates)
    tot_t = sum(dt for _, dt, _ in rates)
    value = tot_n / tot_t
    sample = (f"per step: 2 Vegas iterations x {rates[-1][2]} points of the same workload "
              f"(FP64 oracle, {threads} threads)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / len(rates), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_name(p)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    import paper_1408_6373_gb300 as cg
    from paper_1408_6373_gb300 import workloads as W

    world, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cg.build_library()

    p = W.genz8d4c()
    g = cg.genz(p.ndim, p.families, p.a, p.u)
    # FP32 path with run-time specialisation (CV_JIT): the integrand's families
    # and parameters compiled into the sampling kernel (compiled once, in the
    # warm-up, and cached)
    flags = cg.JIT
    sp = cg.spec(g, nbins=p.nbins, flags=flags, maxeval=p.maxeval, nstart=p.nstart,
                 nincrease=p.nincrease, nbatch=p.nstart)
    samples_per_step = p.maxeval
    ctx = cg.Context(local)
    integ = ctx.integral(sp)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def step():
        integ.reset()
        integ.run()

    # ---- device-timed steps (the clock sampler runs from before the warm-up)
    clocks = clock_sampler(local)
    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    barrier()
    events = []
    clocks.mark_start()
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        step()
        e.record()
        events.append((s, e))
    barrier()
    wall = time.perf_counter() - t0
    clocks.mark_end()
    clk = clocks.stop()
    dev_ms = max_over_ranks(sum(s.elapsed_time(e) for s, e in events), device="cuda")
    res = integ.result()
    value = world * samples_per_step * args.steps / (dev_ms / 1e3)
    launches = integ.kernels_per_run() * args.steps

    # ---- the sampling kernel alone, for the roofline
    edges = torch.tensor(integ.grid(), dtype=torch.float64, device="cuda")
    S1 = torch.zeros(p.ncomp, dtype=torch.float64, device="cuda")
    S2 = torch.zeros_like(S1)
    H = torch.zeros((p.ndim, p.nbins), dtype=torch.float64, device="cuda")
    # the pass as the step runs it: the grid staged once for the FP32 kernel
    table = torch.empty((p.ndim, p.nbins, 2), dtype=torch.float32, device="cuda")
    ctx.stage_grid(p.ndim, p.nbins, flags, edges, table)

    def time_kernel(kflags):
        # the sampling launch alone: the library records CUDA events on its
        # stream immediately around each sampling launch (cv_kernel_timer),
        # so the pass's histogram-partials launch after it is not counted
        for _ in range(3):
            ctx.sample_staged(g, p.nbins, table, 1, p.nstart, kflags, S1, S2, H)
        torch.cuda.synchronize()
        ctx.kernel_timer(True)
        for _ in range(10):
            ctx.sample_staged(g, p.nbins, table, 1, p.nstart, kflags, S1, S2, H)
        ctx.kernel_timer(False)
        times = ctx.kernel_times()
        assert len(times) == 10, times
        return statistics.mean(times)

    k_ms = time_kernel(flags)
    k_ms_generic = time_kernel(0)
    jit_available, jit_compiled = cg.jit_info()
    flops = alg_flops_per_sample(p.ndim, p.families) * p.nstart
    achieved = flops / (k_ms / 1e3) / 1e12
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = sm_count(local)
    peak = fp32_peak_tflops(sm_max, sms)
    # (the committed summary is of the run-time specialised kernel)
    prof = "sampling_specialised_genz8d4c.md" if jit_compiled else None
    traffic = _profile_traffic(prof) if prof else None
    # the bound this kernel actually meets: instruction issue (one warp
    # instruction per cycle per SM sub-partition), with the warp instructions
    # of one launch from the committed ncu summary
    inst = _profile_value(prof, "warp instructions") if prof else None
    issue_peak = sms * 4 * sm_max * 1e6 / 1e9
    issue = None if inst is None else {
        "warp_instructions_per_launch": inst, "achieved": inst / (k_ms / 1e3) / 1e9, "peak": issue_peak,
        "unit": "G warp instructions/s", "frac": inst / (k_ms / 1e3) / 1e9 / issue_peak,
        "peak_basis": f"{sms} SMs x 4 schedulers x 1 instruction per cycle x {sm_max:.0f} MHz"}

    # the FP32 pipe's measured rate (FMA chains), beside the nominal peak
    fma_tflops, fma_ms = ctx.fp32_fma_rate()
    fma = {"value": fma_tflops, "unit": "TFLOP/s", "frac_of_measured": achieved / fma_tflops,
           "basis": f"cv_fp32_fma_rate: 8 independent FMA chains per thread, 4 x 256 threads per SM, "
                    f"one {fma_ms:.1f} ms launch"}

    # ---- end to end through cv_vegas (host description in, host results out)
    h2d, d2h = cg.vegas_io_bytes(p.ndim, p.nbins)
    ctx.vegas(g, flags=flags, maxeval=p.maxeval, nstart=p.nstart, nincrease=p.nincrease, nbins=p.nbins)
    barrier()
    e2e_t = []
    for _ in range(args.steps):
        t = time.perf_counter()
        ctx.vegas(g, flags=flags, maxeval=p.maxeval, nstart=p.nstart, nincrease=p.nincrease,
                  nbins=p.nbins)
        e2e_t.append(time.perf_counter() - t)
    e2e_value = world * samples_per_step / statistics.mean(e2e_t)
    # the same sampling kernel inside whole cv_vegas runs: the sustained
    # figure (the kernel timer makes cv_vegas enqueue its iterations
    # directly, each launch between two events; kept out of the e2e loop)
    ctx.kernel_timer(True)
    for _ in range(max(1, min(args.steps, cg.KERNEL_TIMER_CAP // max(1, p.maxeval // p.nstart)))):
        ctx.vegas(g, flags=flags, maxeval=p.maxeval, nstart=p.nstart, nincrease=p.nincrease,
                  nbins=p.nbins)
    ctx.kernel_timer(False)
    in_run = ctx.kernel_times()
    k_ms_in_run = statistics.mean(in_run) if in_run else None

    # ---- the plain FP64 one-launch-per-iteration comparator
    plain_steps = max(1, min(2, args.steps))
    ctx.vegas(g, flags=cg.FP64 | cg.PLAIN, maxeval=2 * p.nstart, nstart=p.nstart, nbins=p.nbins)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(plain_steps):
        rp = ctx.vegas(g, flags=cg.FP64 | cg.PLAIN, maxeval=p.maxeval, nstart=p.nstart,
                       nbins=p.nbins)
    plain_s = (time.perf_counter() - t) / plain_steps

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": _workload_name(p), "samples_per_step": samples_per_step,
                   "l2": "flushed before every step (256 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": f"sampling kernel, ndim {p.ndim}, FP32, specialised at run time"
                               if jit_compiled else f"k_sample<{p.ndim},float>",
                     "kernel_ms": k_ms, "kernel_ms_generic": k_ms_generic,
                     "kernel_ms_in_vegas_runs": k_ms_in_run, "launches_in_vegas_runs": len(in_run),
                     "jit": {"available": jit_available, "compiled": jit_compiled},
                     "flops_per_sample": alg_flops_per_sample(p.ndim, p.families),
                     "issue": issue, "fma_measured": fma,
                     "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                   f"{sm_max:.0f} MHz (max SM clock, MEASURED_PEAKS.json)"},
        "plain_fp64": {"value": world * samples_per_step / plain_s, "unit": UNIT,
                       "ms_per_step": 1e3 * plain_s,
                       "speedup_of_value": value / (world * samples_per_step / plain_s)},
        "result": {"integral": list(res.integral)[: p.ncomp], "error": list(res.error)[: p.ncomp],
                   "plain_fp64_integral": list(rp.integral)[: p.ncomp],
                   "plain_fp64_error": list(rp.error)[: p.ncomp]},
        "wall_s_timed_region": wall,
    }
    if not args.no_batch:
        line["batch4096"] = measure_batch(ctx, cg, W, args.warmup, args.steps)
    line["gaussian3d"] = measure_gaussian3d(ctx, cg, W)
    line["generators"] = measure_generators(ctx, cg, W)
    line["suave"] = measure_suave(ctx, cg)
    if not args.no_large:
        line["large30d"] = measure_large(ctx, cg, W)
    if not args.no_materialised:
        line["materialised"] = measure_materialised(ctx, cg, W)
    if not args.no_serve:
        line["serve"] = measure_serve(ctx, cg, W, duration=args.serve_seconds)
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, dt, n = cpu_oracle_rate(p, args.cpu_seconds, threads)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                "sample": f"2 Vegas iterations x {n} points of the same workload, "
                                          f"FP64 oracle, {dt:.1f} s"}
        if not args.no_sweep:
            line["cost_sweep"] = measure_cost_sweep(ctx, cg, W, threads)
        line["suave"]["cpu_baseline"] = suave_cpu_rate(threads)
        more = oracle_more_rates(p, W, threads)
        line["cpu_baseline"]["single_thread"] = more["single_thread"]
        for k in ("batch4096", "large30d"):
            if k in line:
                line[k]["cpu_baseline"] = more[k]
        line["accuracy"] = accuracy_leg(line, W, threads)
    if rank == 0:
        line = _strip_private(line)
        line["legs"] = legs_summary(line)  # (last: kept by a tail of the output)
        print(json.dumps(line), flush=True)
    integ.close()
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def measure_batch(ctx, cg, W, warmup: int, steps: int, subset: int = 32) -> dict:
    """The batched persistent path on the 4096-integral workload: device-timed
    runs after autotuning, plus the plain FP64 one-launch-per-iteration
    comparator (host sync per iteration) on a seeded subset of integrals."""
    import torch
    probs = W.batch4096()
    specs = [cg.spec(cg.genz(p.ndim, p.families, p.a, p.u), nbins=p.nbins, maxeval=p.maxeval,
                     nstart=p.nstart, nincrease=p.nincrease) for p in probs]
    samples = sum(p.maxeval for p in probs)
    B = ctx.batch(specs)
    t = time.perf_counter()
    B.autotune()
    tune_s = time.perf_counter() - t
    for _ in range(max(1, warmup // 3)):
        B.run()
    torch.cuda.synchronize()
    ev = []
    for _ in range(max(1, steps // 2)):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        B.run()
        s1.record()
        ev.append((s0, s1))
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    res = B.results()
    launches = B.kernels_per_run()
    tiles = {str(n): B.tile_points(n) for n in (10 ** 4, 10 ** 5, 10 ** 6, 10 ** 7)}
    # (a tile is shared by a CTA's 256 threads)
    ppt = {n: t // 256 for n, t in tiles.items()}
    B.close()
    # plain FP64 comparator on a subset (the full set would take ~30 s)
    idx = list(range(0, len(probs), len(probs) // subset))[:subset]
    sub_samples = sum(probs[i].maxeval for i in idx)
    t = time.perf_counter()
    dev, plain = [], []
    for i in idx:
        p = probs[i]
        rp = ctx.vegas(cg.genz(p.ndim, p.families, p.a, p.u), flags=cg.FP64 | cg.PLAIN,
                       maxeval=p.maxeval, nstart=p.nstart, nbins=p.nbins)
        r = res[i]
        dev.append(abs(r.integral[0] - rp.integral[0]) / max(rp.error[0], 1e-300))
        plain.append((rp.integral[0], rp.error[0]))
    plain_s = time.perf_counter() - t
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    flops = sum(p.maxeval * alg_flops_per_sample(p.ndim, p.families) for p in probs)
    achieved = flops / (ms / 1e3) / 1e12
    sms = sm_count(torch.cuda.current_device())
    peak = fp32_peak_tflops(sm_max, sms)
    # the issue bound, from the committed count of one run's warp instructions
    # (ncu, every class launch) when it was taken on the current sources
    inst = _profile_value("k_batch_sample_batch4096.md", "warp_instructions_per_run")
    issue = None
    if inst:
        issue_peak = sms * 4 * sm_max * 1e6 / 1e9
        issue = {"warp_instructions_per_run": inst, "achieved": inst / (ms / 1e3) / 1e9, "peak": issue_peak,
                 "unit": "G warp instructions/s", "frac": inst / (ms / 1e3) / 1e9 / issue_peak,
                 "flop_frac_at_full_issue": flops / (inst / (issue_peak * 1e9)) / 1e12 / peak,
                 "peak_basis": f"{sms} SMs x 4 schedulers x 1 instruction per cycle x {sm_max:.0f} MHz"}
    return {"workload": "batch4096: 4096 integrals, ndim U{2..16}, family U{0..5}, n/iter "
                        "log-uniform 1e4..1e7, 10 iterations, 64 bins, FP32 eval / FP64 reduce",
            "value": samples / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "issue": issue,
                         "basis": "algorithmic FP32 FLOPs of every integral's samples over the device time "
                                  "of the whole batched run (sampling, refinement and combination)"},
            "_results": [(r.integral[0], r.error[0]) for r in res], "_problems": probs,
            "samples_per_step": samples, "gpu_launches_per_step": launches,
            "autotune_s": tune_s, "tile_points_by_iteration_size": tiles,
            "points_per_thread_by_iteration_size": ppt,
            "plain_fp64_subset": {"integrals": len(idx), "value": sub_samples / plain_s,
                                  "unit": UNIT,
                                  "max_abs_diff_in_sigma": max(dev),
                                  "_results": [(i, plain[k]) for k, i in enumerate(idx)]}}


def measure_materialised(ctx, cg, W) -> dict:
    """The materialised-sample mode on the genz8d4c shape: every iteration's
    1e7 points written to HBM (FP32, dimension-major), evaluated by the
    library's own device integrand, and accumulated.  Reports samples/s and
    the HBM bytes per sample of the library's two kernels (write x, read f;
    the integrand's own traffic, read x and write f, is the caller's)."""
    import torch
    p = W.genz8d4c()
    g = cg.genz(p.ndim, p.families, p.a, p.u)
    ud = cg.GenzCallbackData(g, cg.JIT)  # (the library's integrand, specialised at run time)
    kw = dict(userdata=ud, nvec=p.nstart, flags=0, maxeval=p.maxeval, nstart=p.nstart, nbins=p.nbins)
    ctx.vegas_cb(cg.builtin_integrand(), p.ndim, p.ncomp, **kw)
    torch.cuda.synchronize()
    # device-timed (events on the context's stream around each call) and
    # wall-timed, over three calls
    dev, wall = [], []
    for _ in range(3):
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t = time.perf_counter()
        s0.record()
        r = ctx.vegas_cb(cg.builtin_integrand(), p.ndim, p.ncomp, **kw)
        s1.record()
        torch.cuda.synchronize()
        wall.append(time.perf_counter() - t)
        dev.append(s0.elapsed_time(s1) / 1e3)
    dt = statistics.mean(dev)
    lib_bytes = 4 * p.ndim + 4 * p.ncomp
    all_bytes = 2 * lib_bytes
    rate = p.maxeval / dt
    return {"workload": "genz8d4c with the integrand called on materialised points (nvec = 1e7, "
                        "x and f dimension-major in HBM, library's own Genz integrand specialised at run time)",
            "value": rate, "unit": UNIT, "ms_per_step": 1e3 * dt,
            "wall_ms_per_step": 1e3 * statistics.mean(wall),
            "library_bytes_per_sample": lib_bytes, "all_bytes_per_sample": all_bytes,
            "hbm_gbs_all_kernels": rate * all_bytes / 1e9,
            "hbm_frac_all_kernels": rate * all_bytes / 1e9 / float(measured_peaks().get("hbm_gbs", 6684.8)),
            "integral": list(r.integral), "_results": list(zip(r.integral, r.error))}


def measure_generators(ctx, cg, W, replicates: int = 8) -> dict:
    """genz8d4c (FP32, run-time specialised) with the other point
    generators: scrambled Sobol (randomized QMC: `replicates` independent
    digital shifts; the spread of their results is the RQMC error estimate,
    reported beside Vegas's own error) and pseudo-random Philox points.
    Device-timed samples/s over the replicates."""
    import numpy as np
    import torch
    p = W.genz8d4c()
    g = cg.genz(p.ndim, p.families, p.a, p.u)
    out = {"workload": f"genz8d4c with scrambled Sobol ({replicates} seeds) and pseudo-random points"}
    for name, flag in (("scrambled", cg.SCRAMBLE), ("pseudo", cg.PSEUDO)):
        res, ms = [], 0.0
        for r in range(replicates if flag == cg.SCRAMBLE else 2):
            I = ctx.integral(cg.spec(g, nbins=p.nbins, flags=cg.JIT | flag, maxeval=p.maxeval, nstart=p.nstart,
                                     nincrease=p.nincrease, seed=1000 + r))
            I.reset()
            I.run()  # compiles the specialised kernel once
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            I.reset()
            I.run()
            s1.record()
            torch.cuda.synchronize()
            ms += s0.elapsed_time(s1)
            res.append(I.result())
            I.close()
        ints = np.array([[r.integral[c] for c in range(p.ncomp)] for r in res])
        errs = np.array([[r.error[c] for c in range(p.ncomp)] for r in res])
        out[name] = {"value": len(res) * p.maxeval / (ms * 1e-3), "unit": UNIT,
                     "integral_mean": ints.mean(axis=0).tolist(),
                     "vegas_error": errs.mean(axis=0).tolist()}
        if flag == cg.SCRAMBLE:
            out[name]["rqmc_error"] = (ints.std(axis=0, ddof=1) / math.sqrt(len(res))).tolist()
    return out


def measure_cost_sweep(ctx, cg, W, threads: int, delays=(0, 64, 256, 1024, 4096),
                       cpu_seconds: float = 0.5) -> dict:
    """Integrand cost against speed-up, the GPU counterpart of the paper's
    calibrated-delay experiment (Sect. 4.1, Fig. 1): the Gaussian component of
    genz8d4c with `delay` extra dependent multiply-adds per evaluation (the
    value is unchanged).  Both sides do the same work, one sampling pass on
    the uniform grid: the run-time specialised GPU pass over 1e7 points
    (device-timed) and the oracle on a bounded sample on 1, 4 and all host
    threads (the core-count axis of the paper's figure; part of the
    CPU-baseline leg)."""
    import numpy as np
    import torch

    import oracle as O
    p = W.genz8d4c()
    a, u = np.asarray(p.a)[3:4], np.asarray(p.u)[3:4]
    counts = sorted({1, min(4, threads), threads})
    out = {"workload": "one sampling pass of genz8d4c's Gaussian component (ndim 8, 128 bins, uniform grid) with "
                       "`delay` extra dependent multiply-adds per evaluation: GPU 1e7 points FP32 specialised, "
                       f"oracle FP64 on {counts} host threads", "points": []}
    edges = O.grid_uniform(p.ndim, p.nbins)
    e = torch.tensor(edges, dtype=torch.float64, device="cuda")
    S1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    S2 = torch.zeros_like(S1)
    H = torch.zeros((p.ndim, p.nbins), dtype=torch.float64, device="cuda")
    for dl in delays:
        g = cg.genz(p.ndim, [3], a, u, delay=dl)
        for _ in range(3):
            ctx.sample(g, p.nbins, e, 1, p.nstart, cg.JIT, S1, S2, H)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(5):
            ctx.sample(g, p.nbins, e, 1, p.nstart, cg.JIT, S1, S2, H)
        s1.record()
        torch.cuda.synchronize()
        gpu = 5 * p.nstart / (s0.elapsed_time(s1) * 1e-3)
        prob = O.Problem(p.ndim, [3], a, u, nbins=p.nbins, bits=23, delay=dl)
        cpu = {}
        for th in counts:
            n = 2048 * th
            t = time.perf_counter()
            O.sample(prob, edges, 1, n, nthreads=th)
            dt = time.perf_counter() - t
            n = max(n, int(n * cpu_seconds / max(dt, 1e-3)))
            t = time.perf_counter()
            O.sample(prob, edges, 1, n, nthreads=th)
            cpu[th] = n / (time.perf_counter() - t)
        out["points"].append({"delay": dl, "gpu": gpu, "unit": UNIT,
                              "cpu": {str(th): v for th, v in cpu.items()},
                              "speedup": {str(th): gpu / v for th, v in cpu.items()}})
    return out


SUAVE_PROBLEM = dict(ndim=6, a=[8.0, 6.0, 7.0, 5.0, 9.0, 6.5], u=[0.3, 0.6, 0.45, 0.7, 0.5, 0.35])


def measure_suave(ctx, cg) -> dict:
    """Suave (subregion-adaptive Vegas) on a peaked 6-dimensional Gaussian,
    FP32 (every pass one batched sampling launch over its regions): 32
    splits per round, 2^18 points per region sampling, to relative accuracy
    1e-5; wall time to the result (host decisions and device passes)."""
    import numpy as np
    P = SUAVE_PROBLEM
    g = cg.genz(P["ndim"], [3], np.array([P["a"]]), np.array([P["u"]]))
    kw = dict(nbins=32, flags=0, epsrel=1e-5, maxeval=2 * 10 ** 9, nnew=1 << 18, width=32, max_regions=4096)
    ctx.suave(g, **dict(kw, maxeval=4 << 18))  # first-use costs (kernel attributes, pinned pages)
    t = time.perf_counter()
    r = ctx.suave(g, **kw)
    dt = time.perf_counter() - t
    return {"workload": "suave: Gaussian ndim 6, a = 5..9, FP32 batched passes, 32 bins, 32 splits per round, "
                        "2^18 points per region sampling, epsrel 1e-5",
            "value": r.neval / dt, "unit": UNIT, "seconds": dt, "neval": r.neval, "nregions": r.nregions,
            "fail": r.fail, "integral": float(r.integral[0]), "error": float(r.error[0])}


def suave_cpu_rate(threads: int, budget: int = 1 << 22) -> dict:
    """The oracle's Suave on the same problem and settings with a bounded
    budget (CPU-baseline leg): samples/s on the host's cores."""
    import numpy as np

    import oracle as O
    P = SUAVE_PROBLEM
    prob = O.Problem(P["ndim"], [3], np.array([P["a"]]), np.array([P["u"]]), nbins=32)
    t = time.perf_counter()
    r = O.suave(prob, epsrel=1e-5, maxeval=budget, nnew=1 << 15, width=32, max_regions=4096, nthreads=threads)
    dt = time.perf_counter() - t
    return {"value": r.neval / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"oracle Suave, {r.neval} points (2^15 per region sampling), FP64, {dt:.1f} s"}


def measure_gaussian3d(ctx, cg, W, reps: int = 20) -> dict:
    """The small FP64 case (Gaussian a = 5, u = 1/2, ndim 3, 50 bins,
    10 x 1e4 points): latency-bound, so reported as time per iteration, for
    the graph-replayed integral and the one-launch-per-iteration plain form;
    device-timed, and the result against the closed form."""
    import torch
    p = W.gaussian3d()
    g = cg.genz(p.ndim, p.families, p.a, p.u)
    out = {"workload": "gaussian3d: FP64, Gaussian a = 5, u = 1/2, ndim 3, 50 bins, 10 iterations x 1e4 points"}
    for name, flags in (("graph", cg.FP64), ("plain", cg.FP64 | cg.PLAIN)):
        I = ctx.integral(cg.spec(g, nbins=p.nbins, maxeval=p.maxeval, nstart=p.nstart, flags=flags))
        for _ in range(3):
            I.reset()
            I.run()
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(reps):
            I.reset()
            I.run()
        s1.record()
        torch.cuda.synchronize()
        r = I.result()
        out[f"{name}_us_per_iteration"] = 1e3 * s0.elapsed_time(s1) / (reps * r.iterations)
        I.close()
    exact = (math.sqrt(math.pi) / 5 * math.erf(2.5)) ** 3
    out["integral"], out["error"], out["exact"] = r.integral[0], r.error[0], exact
    return out


def measure_large(ctx, cg, W, steps: int = 1) -> dict:
    """The large single-integral configuration: ndim 30, 256 bins,
    15 iterations x 1e9 points (indices past 2^33), C0 and discontinuous
    integrands, one device-resident integral each with the run-time
    specialised kernel, device-timed."""
    import torch
    out = {"workload": "large30d: ndim 30, C0 and discontinuous, a = 1/2, u ~ U(0,1), 256 bins, "
                       "15 iterations x 1e9 Sobol points, FP32 eval / FP64 reduce"}
    total_ms, total = 0.0, 0
    res = []
    for p in W.large30d():
        g = cg.genz(p.ndim, p.families, p.a, p.u)
        I = ctx.integral(cg.spec(g, nbins=p.nbins, maxeval=p.maxeval, nstart=p.nstart, flags=cg.JIT))
        I.reset()
        I.run()
        torch.cuda.synchronize()
        for _ in range(steps):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            I.reset()
            I.run()
            s1.record()
            torch.cuda.synchronize()
            total_ms += s0.elapsed_time(s1)
            total += p.maxeval
        r = I.result()
        res.append({"family": p.families[0], "integral": r.integral[0], "error": r.error[0], "_p": p})
        I.close()
    out.update({"value": total / (total_ms / 1e3), "unit": UNIT, "ms_per_step": total_ms / steps,
                "samples_per_step": total // steps, "results": res})
    return out


def measure_serve(ctx, cg, W, duration: float = 1.0, rate: float = 2000.0,
                  plain_subset: int = 100) -> dict:
    """The serving loop under Poisson arrivals (ndim U{2..32}, ncomp U{1..4},
    epsrel log-uniform 1e-5..1e-3, maxeval 1e8), submitted in real time; and
    the plain FP64 one-request-at-a-time server on the same arrival times:
    a FIFO queue whose service times are measured on the GPU (cv_vegas with
    CV_FP64 | CV_PLAIN) for the first `plain_subset` requests."""
    reqs = W.serve_requests(rate=rate, duration=duration)
    specs = [cg.spec(cg.genz(p.ndim, p.families, p.a, p.u), nbins=p.nbins, epsrel=p.epsrel,
                     maxeval=p.maxeval, nstart=p.nstart, nincrease=p.nincrease) for _, p in reqs]
    S = ctx.server(hbm_budget_bytes=8 << 30)
    for sp in specs[:8]:  # warm-up: kernel attributes, first launches
        S.wait(S.submit(sp), 600000)
    S.stop()
    S = ctx.server(hbm_budget_bytes=8 << 30)
    ids = []
    t0 = time.perf_counter()
    for (t, _), sp in zip(reqs, specs):
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        ids.append(S.submit(sp))
    res = [S.wait(i, 600000) for i in ids]
    wall = time.perf_counter() - t0
    st = S.stats()
    S.stop()
    samples = sum(r.neval for r in res)
    ok = sum(1 for r in res if r.fail == 0)
    raw = [(p, [(r.integral[c], r.error[c]) for c in range(p.ncomp)], r.neval) for (_, p), r in zip(reqs, res)]
    # the same first requests served alone, at their arrival times: the
    # latency to compare with the plain FP64 server below
    S = ctx.server(hbm_budget_bytes=8 << 30)
    ids = []
    t0 = time.perf_counter()
    for (t, _), sp in zip(reqs[:plain_subset], specs[:plain_subset]):
        now = time.perf_counter() - t0
        if t > now:
            time.sleep(t - now)
        ids.append(S.submit(sp))
    for i in ids:
        S.wait(i, 600000)
    st_sub = S.stats()
    S.stop()
    service = []
    for sp in specs[:plain_subset]:
        t = time.perf_counter()
        ctx.vegas(sp.g, epsrel=sp.epsrel, flags=cg.FP64 | cg.PLAIN, maxeval=sp.maxeval,
                  nstart=sp.nstart, nincrease=sp.nincrease, nbins=sp.nbins)
        service.append(time.perf_counter() - t)
    finish, lat = 0.0, []
    for (t, _), sv in zip(reqs[:plain_subset], service):
        begin = max(t, finish)
        finish = begin + sv
        lat.append(finish - t)
    lat.sort()
    q = lambda p: 1e3 * lat[min(len(lat) - 1, int(p * (len(lat) - 1) + 0.5))]
    return {"workload": f"serve: Poisson {rate:.0f} req/s for {duration:g} s ({len(reqs)} requests), "
                        "ndim U{2..32}, ncomp U{1..4}, Genz families, epsrel log-uniform 1e-5..1e-3, "
                        "maxeval 1e8, nstart 1e4, nincrease 5e4, 64 bins, FP32 eval / FP64 reduce",
            "requests": len(reqs), "reached_accuracy": ok,
            "p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "max_ms": st.max_ms,
            "throughput": {"value": samples / wall, "unit": UNIT},
            "requests_per_s": len(reqs) / wall, "rounds": st.rounds, "max_live": st.max_live,
            "wall_s": wall, "busy_s": st.busy_s, "gpu_s": st.gpu_s,
            "served_first_requests": {"requests": plain_subset, "p50_ms": st_sub.p50_ms,
                                      "p99_ms": st_sub.p99_ms},
            "plain_fp64_fifo": {"requests": len(service), "p50_ms": q(0.5), "p99_ms": q(0.99),
                                "throughput": {"value": sum(r.neval for r in res[:plain_subset]) / sum(service),
                                               "unit": UNIT},
                                "mean_service_ms": 1e3 * sum(service) / len(service)},
            "_results": raw}


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 4096-integral batch")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving run")
    ap.add_argument("--no-materialised", action="store_true", help="skip the materialised-sample run")
    ap.add_argument("--no-sweep", action="store_true", help="skip the integrand-cost sweep")
    ap.add_argument("--no-large", action="store_true", help="skip the 30-dimension 1e9-point run")
    ap.add_argument("--serve-seconds", type=float, default=1.0, help="arrival window of the serving run")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least three untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
