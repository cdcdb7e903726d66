"""Python binding of libcubagpu, the GB300 Vegas sampling library.

Argument marshalling only: every step of the sampling path runs in the CUDA
kernels of the shared library (include/cubagpu.h).  PyTorch tensors serve as
device buffers; the library enqueues on the stream the context was created
with (by default torch's current stream).  If the library has not been
built, the calls raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import weakref
from dataclasses import dataclass

import numpy as np

from .build import LIB as LIB_PATH, build as build_library  # noqa: F401

MAX_DIM = 32
MAX_COMP = 4
MIN_BINS = 2
MAX_BINS = 256
INDEX_LIMIT = 1 << 52
KERNEL_TIMER_CAP = 256

OSCILLATORY, PRODUCT_PEAK, CORNER_PEAK, GAUSSIAN, C0, DISCONTINUOUS, CONST = range(7)
FAMILIES = {"oscillatory": 0, "product_peak": 1, "corner_peak": 2, "gaussian": 3,
            "c0": 4, "discontinuous": 5, "const": 6}

FP64 = 0x100
PLAIN = 0x200
AOS = 0x400
JIT = 0x800
SCRAMBLE = 0x1000  # randomized QMC: Sobol points with a random digital shift per dimension
PSEUDO = 0x2000    # pseudo-random points (Philox4x64-10 keyed by the seed)

OK, EINVAL, ENOMEM, ECUDA, EABORT, ETIMEOUT, EADMIT, EBUSY, ENOTFOUND = 0, -1, -2, -3, -4, -5, -6, -7, -8
ESCRATCH = -9
ENONFINITE = -10
STATIC_SCRATCH_BYTES = 128 * 1024

STREAM_LEGACY = 1  # cudaStreamLegacy


class CubaGpuError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class Genz(ctypes.Structure):
    """cv_genz: one integral of ncomp Genz components in ndim dimensions."""
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("ncomp", ctypes.c_int),
        ("family", ctypes.c_int * MAX_COMP),
        ("a", (ctypes.c_double * MAX_DIM) * MAX_COMP),
        ("u", (ctypes.c_double * MAX_DIM) * MAX_COMP),
        ("delay", ctypes.c_int),
    ]


def genz(ndim: int, families, a, u, delay: int = 0) -> Genz:
    """Build a cv_genz from family ids and [ncomp, ndim] parameter arrays
    (delay: extra dependent multiply-adds per evaluation, a cost knob that
    leaves the values unchanged)."""
    fams = [FAMILIES[f] if isinstance(f, str) else int(f) for f in families]
    nc = len(fams)
    a = np.broadcast_to(np.asarray(a, dtype=np.float64), (nc, ndim))
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), (nc, ndim))
    g = Genz()
    g.ndim, g.ncomp = ndim, nc
    for c in range(nc):
        g.family[c] = fams[c]
        for d in range(ndim):
            g.a[c][d] = float(a[c, d])
            g.u[c][d] = float(u[c, d])
    g.delay = int(delay)
    return g


class Spec(ctypes.Structure):
    """cv_spec: a Vegas problem for a device-resident integral."""
    _fields_ = [
        ("g", Genz),
        ("nbins", ctypes.c_int),
        ("flags", ctypes.c_int),
        ("epsrel", ctypes.c_double),
        ("epsabs", ctypes.c_double),
        ("mineval", ctypes.c_int64),
        ("maxeval", ctypes.c_int64),
        ("nstart", ctypes.c_int64),
        ("nincrease", ctypes.c_int64),
        ("nbatch", ctypes.c_int64),
        ("seed", ctypes.c_uint64),
    ]


class Result(ctypes.Structure):
    """cv_result."""
    _fields_ = [
        ("neval", ctypes.c_int64),
        ("fail", ctypes.c_int),
        ("iterations", ctypes.c_int),
        ("status", ctypes.c_int),
        ("integral", ctypes.c_double * MAX_COMP),
        ("error", ctypes.c_double * MAX_COMP),
        ("prob", ctypes.c_double * MAX_COMP),
        ("chi2", ctypes.c_double * MAX_COMP),
    ]


def spec(g: Genz, nbins=64, flags=0, epsrel=0.0, epsabs=0.0, mineval=0, maxeval=10 ** 6,
         nstart=10 ** 4, nincrease=0, nbatch=1000, seed=0) -> Spec:
    s = Spec()
    s.g = g
    s.nbins, s.flags, s.epsrel, s.epsabs = nbins, flags, epsrel, epsabs
    s.mineval, s.maxeval, s.nstart, s.nincrease, s.nbatch = mineval, maxeval, nstart, nincrease, nbatch
    s.seed = seed
    return s


@dataclass
class SuaveResult:
    nregions: int
    neval: int
    fail: int
    integral: np.ndarray
    error: np.ndarray
    boxes: np.ndarray      # [nregions, ndim, 2] final regions (lo, hi)


class ServerOpts(ctypes.Structure):
    """cv_server_opts."""
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_live", ctypes.c_int),
                ("tile_points", ctypes.c_int)]


class ServeStats(ctypes.Structure):
    """cv_serve_stats."""
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rounds", ctypes.c_int64), ("samples", ctypes.c_int64),
                ("max_live", ctypes.c_int), ("pending", ctypes.c_int),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("wall_s", ctypes.c_double), ("gpu_s", ctypes.c_double)]


_P = ctypes.POINTER
_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_d = ctypes.c_double

INTEGRAND = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                             ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                             ctypes.c_void_p)


class GenzCallbackData(ctypes.Structure):
    """cv_genz_cb_data: userdata of the library's own device integrand."""
    _fields_ = [("g", Genz), ("flags", ctypes.c_int)]


_SIGNATURES = {
    "cv_create": (_i, [_P(_vp), _i, _vp]),
    "cv_destroy": (None, [_vp]),
    "cv_strerror": (ctypes.c_char_p, [_i]),
    "cv_last_error": (ctypes.c_char_p, [_vp]),
    "cv_synchronize": (_i, [_vp]),
    "cv_kernel_timer": (_i, [_vp, _i]),
    "cv_kernel_times": (_i, [_vp, _vp, _i, _P(_i)]),
    "cv_sobol": (_i, [_vp, _i, _u64, _i64, _i, _vp]),
    "cv_points": (_i, [_vp, _i, _u64, _i64, _i, _i, _u64, _vp]),
    "cv_suave": (_i, [_vp, _P(Genz), _i, _i, _u64, ctypes.c_double, ctypes.c_double, _i64, _i64, _i64,
                      ctypes.c_double, _i, _i, _P(_i), _P(_i64), _P(_i), _vp, _vp, _vp]),
    "cv_sample": (_i, [_vp, _P(Genz), _i, _vp, _u64, _i64, _i, _u64, _vp, _vp, _vp]),
    "cv_stage_grid": (_i, [_vp, _i, _i, _i, _vp, _vp]),
    "cv_sample_staged": (_i, [_vp, _P(Genz), _i, _vp, _u64, _i64, _i, _u64, _vp, _vp, _vp]),
    "cv_refine": (_i, [_vp, _i, _i, _vp, _vp]),
    "cv_vegas": (_i, [_vp, _i, _i, _P(Genz), _d, _d, _i, _i, _i64, _i64, _i64, _i64, _i64,
                      _i, _P(_i64), _P(_i), _vp, _vp, _vp]),
    "cv_vegas_io_bytes": (_i, [_i, _i, _P(_i64), _P(_i64)]),
    "cv_fp32_fma_rate": (_i, [_vp, _P(_d), _P(_d)]),
    "cv_jit_info": (_i, [_P(_i), _P(_i)]),
    "cv_jit_check": (_i, [_vp, _i, _i, ctypes.c_char_p, _i]),
    "cv_vegas_noalloc": (_i, [_i, _vp, _i, _i, _P(Genz), _d, _d, _i, _i, _i64, _i64, _i64, _i64,
                              _i64, _i, _P(_i64), _P(_i), _vp, _vp, _vp]),
    "cv_integral_create": (_i, [_vp, _P(Spec), _P(_vp)]),
    "cv_integral_reset": (_i, [_vp]),
    "cv_integral_run": (_i, [_vp]),
    "cv_integral_result": (_i, [_vp, _P(Result)]),
    "cv_integral_grid": (_i, [_vp, _vp]),
    "cv_integral_log": (_i, [_vp, _i, _vp, _vp]),
    "cv_integral_kernels_per_run": (_i, [_vp]),
    "cv_integral_destroy": (None, [_vp]),
    "cv_integral_step": (_i, [_vp, _i]),
    "cv_integral_save": (_i, [_vp, ctypes.c_char_p]),
    "cv_integral_load": (_i, [_vp, ctypes.c_char_p]),
    "cv_integral_check_file": (_i, [_P(Spec), ctypes.c_char_p, ctypes.c_char_p, _i]),
    "cv_integral_set_grid": (_i, [_vp, _vp]),
    "cv_batch_create": (_i, [_vp, _i, _vp, _P(_vp)]),
    "cv_batch_run": (_i, [_vp]),
    "cv_batch_results": (_i, [_vp, _vp]),
    "cv_batch_autotune": (_i, [_vp]),
    "cv_batch_tile_points": (_i, [_vp, ctypes.c_longlong]),
    "cv_batch_kernels_per_run": (_i, [_vp]),
    "cv_batch_log": (_i, [_vp, _i, _i, _vp, _vp]),
    "cv_batch_grid": (_i, [_vp, _i, _vp]),
    "cv_batch_destroy": (None, [_vp]),
    "cv_batch_vegas": (_i, [_vp, _i, _vp, _vp]),
    "cv_vegas_cb": (_i, [_vp, _i, _i, _vp, _vp, _i64, _d, _d, _i, _i, _i64, _i64, _i64, _i64,
                         _i64, _i, _P(_i64), _P(_i), _vp, _vp, _vp]),
    "cv_genz_callback": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "cv_server_start": (_i, [_vp, _P(ServerOpts), _P(_vp)]),
    "cv_submit": (_i, [_vp, _P(Spec), _P(_u64)]),
    "cv_poll": (_i, [_vp, _u64, _P(Result)]),
    "cv_wait": (_i, [_vp, _u64, _i, _P(Result)]),
    "cv_server_stats": (_i, [_vp, _P(ServeStats)]),
    "cv_server_stop": (_i, [_vp]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded shared library (raises if it was never built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with paper_1408_6373_gb300.build_library() "
                "(nvcc, sm_103a); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


def _ptr(t) -> int:
    """Device address of a torch tensor (or an int)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


@dataclass
class VegasResult:
    neval: int
    fail: int
    integral: np.ndarray
    error: np.ndarray
    prob: np.ndarray
    code: int = 0          # the call's return code when it is EABORT or ENONFINITE


class Context:
    """cv_ctx: a device, a stream, and the library's device memory."""

    def __init__(self, device: int = 0, stream=None):
        self._lib = lib()
        if stream is None:
            import torch
            s = torch.cuda.current_stream(device).cuda_stream
            stream = s if s else STREAM_LEGACY
        self._h = ctypes.c_void_p()
        self._children = weakref.WeakSet()
        rc = self._lib.cv_create(ctypes.byref(self._h), device, stream)
        if rc != OK:
            raise CubaGpuError(rc, "cv_create failed: " + self._lib.cv_strerror(rc).decode())

    def close(self):
        if self._h:
            for child in list(self._children):
                child.close()
            self._lib.cv_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, what: str):
        if rc != OK:
            msg = self._lib.cv_last_error(self._h).decode()
            raise CubaGpuError(rc, f"{what}: {msg}")

    def synchronize(self):
        self._check(self._lib.cv_synchronize(self._h), "cv_synchronize")

    def kernel_timer(self, enable: bool):
        """Start (clearing the record) or stop timing the sampling launches."""
        self._check(self._lib.cv_kernel_timer(self._h, 1 if enable else 0), "cv_kernel_timer")

    def kernel_times(self) -> list:
        """Device milliseconds of each timed sampling launch, in order."""
        buf = (ctypes.c_float * KERNEL_TIMER_CAP)()
        n = ctypes.c_int(0)
        self._check(self._lib.cv_kernel_times(self._h, buf, KERNEL_TIMER_CAP, ctypes.byref(n)),
                    "cv_kernel_times")
        return [float(buf[k]) for k in range(min(n.value, KERNEL_TIMER_CAP))]

    # ---------------------------------------------------- building blocks
    def sobol(self, ndim: int, start: int, n: int, bits: int, out):
        """Y[d, j] = X_d(start+j) >> (64-bits) into `out` (int64 [ndim, n])."""
        self._check(self._lib.cv_sobol(self._h, ndim, start, n, bits, _ptr(out)), "cv_sobol")

    def points(self, ndim: int, start: int, n: int, bits: int, flags: int, seed: int, out):
        """cv_points: the coordinates of any point generator (flags 0,
        SCRAMBLE or PSEUDO, keyed by seed) into `out` (int64 [ndim, n])."""
        self._check(self._lib.cv_points(self._h, ndim, start, n, bits, flags, seed, _ptr(out)), "cv_points")

    def sample(self, g: Genz, nbins: int, edges, start: int, n: int, flags: int, S1, S2, H, seed: int = 0):
        """DoSample: add sum J f, sum (J f)^2 and the f^2 histogram of n points."""
        self._check(self._lib.cv_sample(self._h, ctypes.byref(g), nbins, _ptr(edges), start, n,
                                        flags, seed, _ptr(S1), _ptr(S2), _ptr(H)), "cv_sample")

    def stage_grid(self, ndim: int, nbins: int, flags: int, edges, table):
        """cv_stage_grid: the FP32 sampling table of a grid (table: ndim*nbins float2, e.g.
        a float32 tensor of shape [ndim, nbins, 2])."""
        self._check(self._lib.cv_stage_grid(self._h, ndim, nbins, flags, _ptr(edges), _ptr(table)),
                    "cv_stage_grid")

    def sample_staged(self, g: Genz, nbins: int, table, start: int, n: int, flags: int, S1, S2, H,
                      seed: int = 0):
        """cv_sample_staged: sample over a grid table from stage_grid."""
        self._check(self._lib.cv_sample_staged(self._h, ctypes.byref(g), nbins, _ptr(table), start, n,
                                               flags, seed, _ptr(S1), _ptr(S2), _ptr(H)), "cv_sample_staged")

    def suave(self, g: Genz, nbins=16, flags=0, seed=0, epsrel=0.0, epsabs=0.0, mineval=0,
              maxeval=10 ** 5, nnew=1000, flatness=2.0, width=1, max_regions=4096) -> "SuaveResult":
        """cv_suave: subregion-adaptive Vegas (see cubagpu.h for the reading)."""
        nc = g.ncomp
        integral, error = np.zeros(nc), np.zeros(nc)
        boxes = np.zeros((max_regions, g.ndim, 2))
        nreg, neval, fail = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        self._check(self._lib.cv_suave(self._h, ctypes.byref(g), nbins, flags, seed, epsrel, epsabs, mineval,
                                       maxeval, nnew, flatness, width, max_regions, ctypes.byref(nreg),
                                       ctypes.byref(neval), ctypes.byref(fail), integral.ctypes.data,
                                       error.ctypes.data, boxes.ctypes.data), "cv_suave")
        return SuaveResult(nreg.value, neval.value, fail.value, integral, error, boxes[: nreg.value])

    def fp32_fma_rate(self):
        """cv_fp32_fma_rate: measured FP32 FMA rate (TFLOP/s, launch ms)."""
        t, ms = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.cv_fp32_fma_rate(self._h, ctypes.byref(t), ctypes.byref(ms)), "cv_fp32_fma_rate")
        return t.value, ms.value

    def refine(self, ndim: int, nbins: int, H, edges):
        self._check(self._lib.cv_refine(self._h, ndim, nbins, _ptr(H), _ptr(edges)), "cv_refine")

    # ---------------------------------------------------- Vegas
    def vegas(self, g: Genz, epsrel=0.0, epsabs=0.0, flags=0, seed=0, mineval=0,
              maxeval=10 ** 6, nstart=10 ** 4, nincrease=0, nbatch=1000, nbins=64) -> VegasResult:
        nc = g.ncomp
        integral = np.zeros(nc)
        error = np.zeros(nc)
        prob = np.zeros(nc)
        neval, fail = ctypes.c_int64(), ctypes.c_int()
        rc = self._lib.cv_vegas(self._h, g.ndim, nc, ctypes.byref(g), epsrel, epsabs, flags, seed,
                                mineval, maxeval, nstart, nincrease, nbatch, nbins,
                                ctypes.byref(neval), ctypes.byref(fail),
                                integral.ctypes.data, error.ctypes.data, prob.ctypes.data)
        self._check(rc, "cv_vegas")
        return VegasResult(neval.value, fail.value, integral, error, prob)

    def vegas_cb(self, integrand, ndim: int, ncomp: int, userdata=None, nvec=10 ** 6,
                 epsrel=0.0, epsabs=0.0, flags=0, seed=0, mineval=0, maxeval=10 ** 6,
                 nstart=10 ** 4, nincrease=0, nbatch=1000, nbins=64) -> VegasResult:
        """cv_vegas_cb with a device integrand: a ctypes INTEGRAND, an int
        function address (e.g. builtin_integrand()), or a Python callable
        f(x, fvals, nvec, stream) -> int receiving torch views of the device
        buffers (x: [ndim, nvec], fvals: [ncomp, nvec]; CV_AOS: transposed)."""
        if isinstance(integrand, int):
            fn = ctypes.cast(integrand, INTEGRAND)
        elif isinstance(integrand, INTEGRAND):
            fn = integrand
        else:
            fn = _torch_integrand(integrand, flags)
        nc = ncomp
        integral, error, prob = np.zeros(nc), np.zeros(nc), np.zeros(nc)
        neval, fail = ctypes.c_int64(), ctypes.c_int()
        ud = ctypes.cast(ctypes.pointer(userdata), ctypes.c_void_p) if userdata is not None else None
        rc = self._lib.cv_vegas_cb(self._h, ndim, nc, ctypes.cast(fn, ctypes.c_void_p), ud, nvec,
                                   epsrel, epsabs, flags, seed, mineval, maxeval, nstart,
                                   nincrease, nbatch, nbins, ctypes.byref(neval), ctypes.byref(fail),
                                   integral.ctypes.data, error.ctypes.data, prob.ctypes.data)
        if rc in (EABORT, ENONFINITE):
            return VegasResult(neval.value, fail.value, integral, error, prob, rc)
        self._check(rc, "cv_vegas_cb")
        return VegasResult(neval.value, fail.value, integral, error, prob)

    def integral(self, sp: Spec) -> "Integral":
        return Integral(self, sp)

    def server(self, hbm_budget_bytes=0, max_live=0, tile_points=0) -> "Server":
        return Server(self, hbm_budget_bytes, max_live, tile_points)

    def batch(self, specs) -> "Batch":
        return Batch(self, specs)

    def batch_vegas(self, specs):
        """cv_batch_vegas: run every spec together; list of Result."""
        arr = (Spec * len(specs))(*specs)
        res = (Result * len(specs))()
        self._check(self._lib.cv_batch_vegas(self._h, len(specs), arr, res), "cv_batch_vegas")
        return list(res)


def vegas_noalloc(g: Genz, device: int = 0, stream=None, epsrel=0.0, epsabs=0.0, flags=0,
                  seed=0, mineval=0, maxeval=10 ** 6, nstart=10 ** 4, nincrease=0, nbatch=1000,
                  nbins=64) -> VegasResult:
    """cv_vegas_noalloc: the Vegas call for callers that cannot allocate
    device memory (scratch in a static device array; see cubagpu.h).
    `stream` defaults to torch's current stream on `device`."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(device).cuda_stream or None
    nc = g.ncomp
    integral, error, prob = np.zeros(nc), np.zeros(nc), np.zeros(nc)
    neval, fail = ctypes.c_int64(), ctypes.c_int()
    rc = lib().cv_vegas_noalloc(device, stream, g.ndim, nc, ctypes.byref(g), epsrel, epsabs,
                                flags, seed, mineval, maxeval, nstart, nincrease, nbatch, nbins,
                                ctypes.byref(neval), ctypes.byref(fail), integral.ctypes.data,
                                error.ctypes.data, prob.ctypes.data)
    if rc != OK:
        raise CubaGpuError(rc, "cv_vegas_noalloc: " + lib().cv_strerror(rc).decode())
    return VegasResult(neval.value, fail.value, integral, error, prob)


def check_state_file(sp: Spec, path: str):
    """cv_integral_check_file: (ok, reason) for a file written by
    Integral.save, checked against the problem sp on the host alone."""
    buf = ctypes.create_string_buffer(512)
    rc = lib().cv_integral_check_file(ctypes.byref(sp), os.fsencode(path), buf, len(buf))
    return rc == OK, buf.value.decode(errors="replace")


def jit_info():
    """(available, compiled): can kernels be specialised at run time, and how
    many have been in this process (CV_JIT)."""
    a, c = ctypes.c_int(), ctypes.c_int()
    lib().cv_jit_info(ctypes.byref(a), ctypes.byref(c))
    return bool(a.value), c.value


def jit_check(g: Genz, nbins: int, flags: int = 0):
    """cv_jit_check: compile, without loading, the specialised kernel CV_JIT
    would build for g, nbins and the generator of flags.  Returns (ok, reason)."""
    buf = ctypes.create_string_buffer(512)
    rc = lib().cv_jit_check(ctypes.byref(g), nbins, flags, buf, len(buf))
    if rc == EINVAL:
        raise CubaGpuError(rc, "cv_jit_check")
    return rc == OK, buf.value.decode(errors="replace")


def vegas_io_bytes(ndim: int, nbins: int):
    h2d, d2h = ctypes.c_int64(), ctypes.c_int64()
    rc = lib().cv_vegas_io_bytes(ndim, nbins, ctypes.byref(h2d), ctypes.byref(d2h))
    if rc != OK:
        raise CubaGpuError(rc, "cv_vegas_io_bytes")
    return h2d.value, d2h.value


class Integral:
    """cv_integral: one Vegas problem whose state stays on the device."""

    def __init__(self, ctx: Context, sp: Spec):
        self.ctx = ctx
        self.spec = sp
        self._h = ctypes.c_void_p()
        ctx._check(ctx._lib.cv_integral_create(ctx._h, ctypes.byref(sp), ctypes.byref(self._h)),
                   "cv_integral_create")
        ctx._children.add(self)

    def close(self):
        if self._h:
            if self.ctx._h:
                self.ctx._lib.cv_integral_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        self.ctx._check(self.ctx._lib.cv_integral_reset(self._h), "cv_integral_reset")

    def run(self):
        self.ctx._check(self.ctx._lib.cv_integral_run(self._h), "cv_integral_run")

    def result(self) -> Result:
        r = Result()
        self.ctx._check(self.ctx._lib.cv_integral_result(self._h, ctypes.byref(r)),
                        "cv_integral_result")
        return r

    def grid(self) -> np.ndarray:
        e = np.zeros((self.spec.g.ndim, self.spec.nbins + 1))
        self.ctx._check(self.ctx._lib.cv_integral_grid(self._h, e.ctypes.data), "cv_integral_grid")
        return e

    def log(self, max_iter: int):
        nc = self.spec.g.ncomp
        I = np.zeros((max_iter, nc))
        V = np.zeros((max_iter, nc))
        self.ctx._check(self.ctx._lib.cv_integral_log(self._h, max_iter, I.ctypes.data,
                                                      V.ctypes.data), "cv_integral_log")
        return I, V

    def kernels_per_run(self) -> int:
        return self.ctx._lib.cv_integral_kernels_per_run(self._h)

    def step(self, max_iter: int):
        self.ctx._check(self.ctx._lib.cv_integral_step(self._h, max_iter), "cv_integral_step")

    def save(self, path: str):
        self.ctx._check(self.ctx._lib.cv_integral_save(self._h, os.fsencode(path)), "cv_integral_save")

    def load(self, path: str):
        self.ctx._check(self.ctx._lib.cv_integral_load(self._h, os.fsencode(path)), "cv_integral_load")

    def set_grid(self, edges: np.ndarray):
        e = np.ascontiguousarray(edges, dtype=np.float64)
        self.ctx._check(self.ctx._lib.cv_integral_set_grid(self._h, e.ctypes.data), "cv_integral_set_grid")


class Batch:
    """cv_batch: many Vegas integrals run together from one CUDA graph."""

    def __init__(self, ctx: Context, specs):
        self.ctx = ctx
        self.count = len(specs)
        self._specs = (Spec * self.count)(*specs)
        self._h = ctypes.c_void_p()
        ctx._check(ctx._lib.cv_batch_create(ctx._h, self.count, self._specs, ctypes.byref(self._h)),
                   "cv_batch_create")
        ctx._children.add(self)

    def close(self):
        if self._h:
            if self.ctx._h:
                self.ctx._lib.cv_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self):
        self.ctx._check(self.ctx._lib.cv_batch_run(self._h), "cv_batch_run")

    def autotune(self):
        self.ctx._check(self.ctx._lib.cv_batch_autotune(self._h), "cv_batch_autotune")

    def results(self):
        res = (Result * self.count)()
        self.ctx._check(self.ctx._lib.cv_batch_results(self._h, res), "cv_batch_results")
        return list(res)

    def tile_points(self, n: int) -> int:
        """Points per tile for an iteration of n points."""
        return self.ctx._lib.cv_batch_tile_points(self._h, n)

    def kernels_per_run(self) -> int:
        return self.ctx._lib.cv_batch_kernels_per_run(self._h)

    def log(self, item: int, max_iter: int):
        """cv_batch_log: (I[m, ncomp], var[m, ncomp]) of integral `item`."""
        nc = self._specs[item].g.ncomp
        lI = np.zeros((max_iter, nc))
        lV = np.zeros((max_iter, nc))
        self.ctx._check(self.ctx._lib.cv_batch_log(self._h, item, max_iter, lI.ctypes.data, lV.ctypes.data),
                        "cv_batch_log")
        return lI, lV

    def grid(self, item: int) -> np.ndarray:
        """cv_batch_grid: the current edges [ndim, nbins+1] of integral `item`."""
        sp = self._specs[item]
        e = np.zeros((sp.g.ndim, sp.nbins + 1))
        self.ctx._check(self.ctx._lib.cv_batch_grid(self._h, item, e.ctypes.data), "cv_batch_grid")
        return e


class Server:
    """cv_server: continuous-batching request loop on the device."""

    def __init__(self, ctx: Context, hbm_budget_bytes=0, max_live=0, tile_points=0):
        self.ctx = ctx
        o = ServerOpts(hbm_budget_bytes, max_live, tile_points)
        self._h = ctypes.c_void_p()
        ctx._check(ctx._lib.cv_server_start(ctx._h, ctypes.byref(o), ctypes.byref(self._h)),
                   "cv_server_start")
        ctx._children.add(self)

    def submit(self, sp: Spec) -> int:
        rid = ctypes.c_uint64()
        self.ctx._check(self.ctx._lib.cv_submit(self._h, ctypes.byref(sp), ctypes.byref(rid)),
                        "cv_submit")
        return rid.value

    def poll(self, rid: int):
        """Result, or None while the request runs."""
        r = Result()
        rc = self.ctx._lib.cv_poll(self._h, rid, ctypes.byref(r))
        if rc == EBUSY:
            return None
        self.ctx._check(rc, "cv_poll")
        return r

    def wait(self, rid: int, timeout_ms: int = 60000) -> Result:
        r = Result()
        self.ctx._check(self.ctx._lib.cv_wait(self._h, rid, timeout_ms, ctypes.byref(r)), "cv_wait")
        return r

    def stats(self) -> ServeStats:
        st = ServeStats()
        self.ctx._check(self.ctx._lib.cv_server_stats(self._h, ctypes.byref(st)), "cv_server_stats")
        return st

    def stop(self):
        if self._h:
            h, self._h = self._h, ctypes.c_void_p()
            if self.ctx._h:
                self.ctx._check(self.ctx._lib.cv_server_stop(h), "cv_server_stop")

    close = stop

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def builtin_integrand() -> int:
    """Address of cv_genz_callback, the library's device integrand (its
    userdata is a GenzCallbackData)."""
    return ctypes.cast(lib().cv_genz_callback, ctypes.c_void_p).value


class _DeviceBuffer:
    """__cuda_array_interface__ view of a device pointer for torch."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"data": (ptr, False), "shape": shape,
                                         "typestr": typestr, "version": 3, "strides": None}


def _torch_integrand(fn, flags):
    import torch
    typestr = "<f8" if flags & FP64 else "<f4"

    def tramp(ndim_p, x, ncomp_p, f, userdata, nvec_p, ld_p, stream):
        ndim, ncomp, nvec, ld = ndim_p[0], ncomp_p[0], nvec_p[0], ld_p[0]
        if flags & AOS:
            xv = torch.as_tensor(_DeviceBuffer(x, (nvec, ndim), typestr), device="cuda")
            fv = torch.as_tensor(_DeviceBuffer(f, (nvec, ncomp), typestr), device="cuda")
        else:
            xv = torch.as_tensor(_DeviceBuffer(x, (ndim, ld), typestr), device="cuda")[:, :nvec]
            fv = torch.as_tensor(_DeviceBuffer(f, (ncomp, ld), typestr), device="cuda")[:, :nvec]
        return int(fn(xv, fv, nvec, stream))

    cb = INTEGRAND(tramp)
    _KEEP.append(cb)
    return cb


_KEEP = []
