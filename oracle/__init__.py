"""FP64 CPU oracle for the Vegas sampling path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never imports it, and it imports nothing from the product.

The arithmetic lives in ``cuba_oracle.c`` (plain C, FP64, Neumaier sums);
this module compiles it with gcc, loads it through ctypes and marshals
numpy arrays.  The Sobol direction numbers are derived here from the
Joe-Kuo primitive polynomials and initial numbers that scipy ships
(``new-joe-kuo-6.21201``), by the Bratley-Fox recurrence in the C file.

Every function is pinned by a test against something other than itself:
scipy's unscrambled Sobol points, the digital (0,m,2)-net property, Genz
closed forms checked against independent quadrature, and exact special
cases (f = 1, equal histograms).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cuba_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

MAX_DIM = 64
MAX_COMP = 8
MAX_BINS = 256

OSCILLATORY, PRODUCT_PEAK, CORNER_PEAK, GAUSSIAN, C0, DISCONTINUOUS, CONST = range(7)
FAMILY_NAMES = ["oscillatory", "product_peak", "corner_peak", "gaussian", "c0",
                "discontinuous", "const"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (ISO C11, no FP contraction, so x86 and Arm
    round identically) and return the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("ncomp", ctypes.c_int),
        ("nbins", ctypes.c_int),
        ("bits", ctypes.c_int),
        ("band_bits", ctypes.c_int),
        ("family", ctypes.c_int * MAX_COMP),
        ("a", (ctypes.c_double * MAX_DIM) * MAX_COMP),
        ("u", (ctypes.c_double * MAX_DIM) * MAX_COMP),
        ("gen", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("delay", ctypes.c_int),
    ]


_P = ctypes.POINTER
_d = ctypes.c_double
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_int = ctypes.c_int
_vp = ctypes.c_void_p


def _bind(lib):
    sig = {
                "or_sobol_directions": (_int, [_int, _vp, _vp, _int, _vp]),
                "or_sobol_word": (None, [_int, _vp, _u64, _vp]),
                "or_sobol_coords": (_int, [_int, _vp, _u64, _i64, _int, _vp]),
                "or_philox4x64": (None, [_vp, _vp, _vp]),
                "or_point_words": (None, [_int, _u64, _int, _vp, _u64, _vp]),
                "or_point_coords": (_int, [_int, _u64, _int, _vp, _u64, _i64, _int, _vp]),
                "or_suave": (_int, [_P(_Problem), _vp, _d, _d, _i64, _i64, _i64, _d, _int, _int, _int,
                                    _P(_int), _P(_i64), _P(_int), _vp, _vp, _vp]),
                "or_grid_uniform": (None, [_int, _int, _vp]),
                "or_map": (_d, [_int, _int, _vp, _vp, _int, _vp, _vp]),
                "or_genz": (_d, [_int, _int, _vp, _vp, _vp]),
                "or_genz_exact": (_d, [_int, _int, _vp, _vp]),
                "or_corner_peak_incl_excl": (_d, [_int, _vp]),
                "or_sample": (_int, [_P(_Problem), _vp, _vp, _u64, _i64, _int,
                                     _vp, _vp, _vp]),
                "or_sample_bounds": (_int, [_P(_Problem), _vp, _vp, _u64, _i64, _int,
                                            _vp, _vp, _vp, _vp, _vp, _vp]),
                "or_refine": (None, [_int, _int, _vp, _vp]),
                "or_rebin": (None, [_int, _int, _vp, _vp]),
                "or_chi2_cdf": (_d, [_d, _int]),
                "or_combine": (None, [_int, _vp, _vp, _P(_d), _P(_d), _P(_d), _P(_d)]),
                "or_vegas": (_int, [_P(_Problem), _vp, _d, _d, _i64, _i64, _i64,
                                    _i64, _int, _vp, _P(_i64), _P(_int), _P(_int),
                                    _vp, _vp, _vp, _vp, _int, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def compile_variant(source_text: str, path: str) -> str:
    """Compile another version of the oracle's C source (the tests plant
    mistakes in copies to show that the pins catch them)."""
    src = path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", path, src, "-lm", "-lpthread"])
    return path


class use_library:
    """Context manager: route every oracle call to the library at `path`."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        with _lock:
            self._saved = _lib
            _lib = _bind(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self._saved


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Sobol
# --------------------------------------------------------------------------
_joe_kuo = None


def joe_kuo_table():
    """(poly, vinit) of the Joe-Kuo direction numbers as scipy ships them:
    poly[d] is the primitive polynomial of dimension d as an integer (bit j =
    coefficient of x^j), vinit[d, :deg] its initial odd numbers m_1..m_s."""
    global _joe_kuo
    if _joe_kuo is None:
        import scipy.stats._sobol as _s
        z = np.load(os.path.join(os.path.dirname(_s.__file__),
                                 "_sobol_direction_numbers.npz"))
        _joe_kuo = (np.ascontiguousarray(z["poly"][:MAX_DIM], dtype=np.int64),
                    np.ascontiguousarray(z["vinit"][:MAX_DIM], dtype=np.int64))
    return _joe_kuo


def sobol_directions(ndim: int, poly=None, vinit=None) -> np.ndarray:
    """64-bit direction words V[d, k] = m_{d,k+1} << (63-k), shape [ndim, 64]."""
    if poly is None:
        poly, vinit = joe_kuo_table()
    poly = np.ascontiguousarray(poly, dtype=np.int64)
    vinit = np.ascontiguousarray(vinit, dtype=np.int64)
    V = np.zeros((ndim, 64), dtype=np.uint64)
    rc = _load().or_sobol_directions(ndim, _ptr(poly), _ptr(vinit), vinit.shape[1], _ptr(V))
    if rc != 0:
        raise ValueError("bad direction-number input")
    return V


def sobol_words(ndim: int, indices, V=None) -> np.ndarray:
    """Full 64-bit Sobol words X_d(i), shape [ndim, len(indices)]."""
    V = sobol_directions(ndim) if V is None else V
    idx = np.asarray(indices, dtype=np.uint64)
    out = np.zeros((ndim, idx.size), dtype=np.uint64)
    X = np.zeros(ndim, dtype=np.uint64)
    lib = _load()
    for j, i in enumerate(idx):
        lib.or_sobol_word(ndim, _ptr(V), int(i), _ptr(X))
        out[:, j] = X
    return out


def sobol_coords(ndim: int, start: int, n: int, bits: int, V=None) -> np.ndarray:
    """y-coordinates Y[d, j] = X_d(start+j) >> (64-bits) (integers)."""
    V = sobol_directions(ndim) if V is None else V
    Y = np.zeros((ndim, n), dtype=np.uint64)
    rc = _load().or_sobol_coords(ndim, _ptr(V), start, n, bits, _ptr(Y))
    if rc != 0:
        raise ValueError("bad arguments")
    return Y


SOBOL, SCRAMBLED, PSEUDO = 0, 1, 2


def philox(ctr, key) -> np.ndarray:
    """Philox4x64-10 block of counter ctr[4] under key[2] (uint64)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().or_philox4x64(_ptr(c), _ptr(k), _ptr(out))
    return out


def point_words(gen: int, seed: int, ndim: int, indices, V=None) -> np.ndarray:
    """64-bit words of any generator, shape [ndim, len(indices)]."""
    V = sobol_directions(ndim) if V is None else V
    idx = np.asarray(indices, dtype=np.uint64)
    out = np.zeros((ndim, idx.size), dtype=np.uint64)
    X = np.zeros(ndim, dtype=np.uint64)
    lib = _load()
    for j, i in enumerate(idx):
        lib.or_point_words(gen, seed, ndim, _ptr(V), int(i), _ptr(X))
        out[:, j] = X
    return out


def point_coords(gen: int, seed: int, ndim: int, start: int, n: int, bits: int, V=None) -> np.ndarray:
    """y-coordinates of any generator, [ndim, n] integers."""
    V = sobol_directions(ndim) if V is None else V
    Y = np.zeros((ndim, n), dtype=np.uint64)
    rc = _load().or_point_coords(gen, seed, ndim, _ptr(V), start, n, bits, _ptr(Y))
    if rc != 0:
        raise ValueError("bad arguments")
    return Y


# --------------------------------------------------------------------------
# Grid, integrands
# --------------------------------------------------------------------------
def grid_uniform(ndim: int, nbins: int) -> np.ndarray:
    e = np.zeros((ndim, nbins + 1), dtype=np.float64)
    _load().or_grid_uniform(ndim, nbins, _ptr(e))
    return e


def map_point(edges: np.ndarray, Y, bits: int):
    """Map one point's y-integers through the grid: (x[ndim], J, k[ndim])."""
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    ndim, n1 = edges.shape
    Y = np.ascontiguousarray(Y, dtype=np.uint64)
    x = np.zeros(ndim)
    k = np.zeros(ndim, dtype=np.int32)
    J = _load().or_map(ndim, n1 - 1, _ptr(edges), _ptr(Y), bits, _ptr(x), _ptr(k))
    return x, J, k


def genz(family: int, a, u, x) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return _load().or_genz(family, a.size, _ptr(a), _ptr(u), _ptr(x))


def genz_exact(family: int, a, u) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    return _load().or_genz_exact(family, a.size, _ptr(a), _ptr(u))


def corner_peak_incl_excl(a) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return _load().or_corner_peak_incl_excl(a.size, _ptr(a))


# --------------------------------------------------------------------------
# Problems, sampling, refinement, combination, Vegas
# --------------------------------------------------------------------------
@dataclass
class Problem:
    """One integral: ncomp Genz components over [0,1]^ndim."""
    ndim: int
    family: list
    a: np.ndarray          # [ncomp, ndim]
    u: np.ndarray          # [ncomp, ndim]
    nbins: int = 50
    bits: int = 52         # fraction bits of y: 52 (FP64 path) or 23 (FP32 path)
    # significand bits of the evaluation a pass is compared with, for the
    # discontinuity band of sample_bounds: None = 24 (binary32) when
    # bits == 23, else 0 (no band: an FP64 evaluation decides as the oracle)
    band_bits: int = None
    gen: int = 0           # point generator: SOBOL, SCRAMBLED or PSEUDO
    seed: int = 0          # Philox key of the scrambled and pseudo-random generators
    delay: int = 0         # integrand-cost knob (extra multiply-adds per evaluation)
    V: np.ndarray = field(default=None, repr=False)

    @property
    def ncomp(self) -> int:
        return len(self.family)

    def _c(self) -> _Problem:
        p = _Problem()
        p.ndim, p.ncomp, p.nbins, p.bits = self.ndim, self.ncomp, self.nbins, self.bits
        bb = self.band_bits
        p.band_bits = int(bb) if bb is not None else (24 if self.bits == 23 else 0)
        p.gen, p.seed, p.delay = int(self.gen), int(self.seed), int(self.delay)
        a = np.asarray(self.a, dtype=np.float64).reshape(self.ncomp, self.ndim)
        u = np.asarray(self.u, dtype=np.float64).reshape(self.ncomp, self.ndim)
        for c in range(self.ncomp):
            p.family[c] = int(self.family[c])
            for d in range(self.ndim):
                p.a[c][d] = a[c, d]
                p.u[c][d] = u[c, d]
        return p

    def directions(self) -> np.ndarray:
        if self.V is None:
            self.V = sobol_directions(self.ndim)
        return self.V

    def exact(self) -> np.ndarray:
        a = np.asarray(self.a, dtype=np.float64).reshape(self.ncomp, self.ndim)
        u = np.asarray(self.u, dtype=np.float64).reshape(self.ncomp, self.ndim)
        return np.array([genz_exact(int(self.family[c]), a[c], u[c])
                         for c in range(self.ncomp)])


def sample(prob: Problem, edges: np.ndarray, start: int, n: int, nthreads: int = 1):
    """One sampling pass: (S1[ncomp], S2[ncomp], H[ndim, nbins])."""
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    S1 = np.zeros(prob.ncomp)
    S2 = np.zeros(prob.ncomp)
    H = np.zeros((prob.ndim, prob.nbins))
    p = prob._c()
    rc = _load().or_sample(ctypes.byref(p), _ptr(prob.directions()), _ptr(edges),
                           start, n, nthreads, _ptr(S1), _ptr(S2), _ptr(H))
    if rc != 0:
        raise ValueError(f"or_sample failed ({rc})")
    return S1, S2, H


@dataclass
class PassBounds:
    """One sampling pass with what bounds a lower-precision evaluation of it:
    A1[c] = sum |J f_c|; B1[c], B2[c] the boundary mass of the discontinuity
    band (points a binary32 evaluation may decide either way, see the C
    source): such an evaluation may differ by up to B1 in S1, B2 in S2 and
    B2[0] in any histogram bin."""
    S1: np.ndarray
    S2: np.ndarray
    H: np.ndarray
    A1: np.ndarray
    B1: np.ndarray
    B2: np.ndarray


def sample_bounds(prob: Problem, edges: np.ndarray, start: int, n: int,
                  nthreads: int = 1) -> PassBounds:
    """sample() plus sum |J f| and the boundary mass of the pass."""
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    nc = prob.ncomp
    out = [np.zeros(nc) for _ in range(5)]
    H = np.zeros((prob.ndim, prob.nbins))
    p = prob._c()
    S1, S2, A1, B1, B2 = out
    rc = _load().or_sample_bounds(ctypes.byref(p), _ptr(prob.directions()), _ptr(edges),
                                  start, n, nthreads, _ptr(S1), _ptr(S2), _ptr(H),
                                  _ptr(A1), _ptr(B1), _ptr(B2))
    if rc != 0:
        raise ValueError(f"or_sample_bounds failed ({rc})")
    return PassBounds(S1, S2, H, A1, B1, B2)


def refine(edges: np.ndarray, H: np.ndarray) -> np.ndarray:
    """Refined copy of the grid `edges` [ndim, N+1] from the histogram H."""
    e = np.array(edges, dtype=np.float64, copy=True, order="C")
    H = np.ascontiguousarray(H, dtype=np.float64)
    ndim, n1 = e.shape
    _load().or_refine(ndim, n1 - 1, _ptr(H), _ptr(e))
    return e


def rebin(edges: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Rebinned copy of `edges` [ndim, N+1] for bin weights r [ndim, N]."""
    e = np.array(edges, dtype=np.float64, copy=True, order="C")
    r = np.ascontiguousarray(r, dtype=np.float64)
    ndim, n1 = e.shape
    _load().or_rebin(ndim, n1 - 1, _ptr(r), _ptr(e))
    return e


def chi2_cdf(x: float, dof: int) -> float:
    return _load().or_chi2_cdf(x, dof)


def combine(I, var):
    """(mean, err, chi2, prob) of iteration results I[j], var[j]."""
    I = np.ascontiguousarray(I, dtype=np.float64)
    var = np.ascontiguousarray(var, dtype=np.float64)
    out = [ctypes.c_double() for _ in range(4)]
    _load().or_combine(I.size, _ptr(I), _ptr(var), *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


def iteration_result(S1, S2, n):
    """I = S1/n, var = (S2/n - I^2)/(n-1) per component."""
    I = np.asarray(S1) / n
    return I, (np.asarray(S2) / n - I * I) / (n - 1)


@dataclass
class VegasResult:
    neval: int
    fail: int
    niter: int
    integral: np.ndarray
    error: np.ndarray
    chi2: np.ndarray
    prob: np.ndarray
    edges: np.ndarray
    iter_I: np.ndarray
    iter_var: np.ndarray


def vegas(prob: Problem, epsrel=0.0, epsabs=0.0, mineval=0, maxeval=10**4,
          nstart=1000, nincrease=0, nthreads=1, edges=None, max_log=4096) -> VegasResult:
    e = grid_uniform(prob.ndim, prob.nbins) if edges is None else \
        np.array(edges, dtype=np.float64, copy=True, order="C")
    nc = prob.ncomp
    out = {k: np.zeros(nc) for k in ("integral", "error", "chi2", "prob")}
    iI = np.zeros((max_log, nc))
    iV = np.zeros((max_log, nc))
    neval, fail, niter = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int()
    p = prob._c()
    rc = _load().or_vegas(ctypes.byref(p), _ptr(prob.directions()), epsrel, epsabs,
                          mineval, maxeval, nstart, nincrease, nthreads, _ptr(e),
                          ctypes.byref(neval), ctypes.byref(fail), ctypes.byref(niter),
                          _ptr(out["integral"]), _ptr(out["error"]), _ptr(out["chi2"]),
                          _ptr(out["prob"]), max_log, _ptr(iI), _ptr(iV))
    if rc != 0:
        raise ValueError(f"or_vegas failed ({rc})")
    m = niter.value
    return VegasResult(neval.value, fail.value, m, out["integral"], out["error"],
                       out["chi2"], out["prob"], e, iI[:m], iV[:m])


@dataclass
class SuaveResult:
    nregions: int
    neval: int
    fail: int
    integral: np.ndarray
    error: np.ndarray
    boxes: np.ndarray      # [nregions, ndim, 2] final regions (lo, hi)


def suave(prob: Problem, epsrel=0.0, epsabs=0.0, mineval=0, maxeval=10 ** 5, nnew=1000,
          flatness=2.0, width=1, max_regions=4096, nthreads=1) -> SuaveResult:
    """Suave (subregion-adaptive Vegas) as read in the C source."""
    nc = prob.ncomp
    integral, error = np.zeros(nc), np.zeros(nc)
    boxes = np.zeros((max_regions, prob.ndim, 2))
    nreg, neval, fail = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
    p = prob._c()
    rc = _load().or_suave(ctypes.byref(p), _ptr(prob.directions()), epsrel, epsabs, mineval, maxeval,
                          nnew, flatness, width, max_regions, nthreads, ctypes.byref(nreg),
                          ctypes.byref(neval), ctypes.byref(fail), _ptr(integral), _ptr(error), _ptr(boxes))
    if rc != 0:
        raise ValueError(f"or_suave failed ({rc})")
    return SuaveResult(nreg.value, neval.value, fail.value, integral, error, boxes[: nreg.value])
