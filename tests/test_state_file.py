"""The checks a saved integral state passes before cv_integral_load copies
it to the device, run on the host alone through cv_integral_check_file (no
GPU): a well-formed state of the problem is accepted, and each kind of
damage -- truncation, trailing bytes, another problem, a broken grid or
histogram, counters off the schedule -- is refused with its reason.

The files are written here from the library's documented layout: a
problem header, the device state record, the grid edges [ndim][nbins+1],
the histogram [ndim][nbins] and the iteration log (256 x 4 integrals, then
256 x 4 variances).  The mirrors below must match the library's structs:
the header carries the state record's size, so a mirror that drifts makes
the well-formed case fail."""
import ctypes

import numpy as np
import pytest

import paper_1408_6373_gb300 as cg

LOG_CAP = 256


class Header(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_char * 8), ("version", ctypes.c_uint), ("state_bytes", ctypes.c_uint),
                ("ndim", ctypes.c_int), ("ncomp", ctypes.c_int), ("nbins", ctypes.c_int), ("flags", ctypes.c_int),
                ("family", ctypes.c_int * cg.MAX_COMP),
                ("a", (ctypes.c_double * cg.MAX_DIM) * cg.MAX_COMP),
                ("u", (ctypes.c_double * cg.MAX_DIM) * cg.MAX_COMP),
                ("epsrel", ctypes.c_double), ("epsabs", ctypes.c_double),
                ("mineval", ctypes.c_longlong), ("maxeval", ctypes.c_longlong),
                ("nstart", ctypes.c_longlong), ("nincrease", ctypes.c_longlong),
                ("seed", ctypes.c_ulonglong)]


_D4 = ctypes.c_double * cg.MAX_COMP


class State(ctypes.Structure):
    _fields_ = [("next_index", ctypes.c_ulonglong), ("n_cur", ctypes.c_longlong), ("neval", ctypes.c_longlong),
                ("iter", ctypes.c_int), ("stopped", ctypes.c_int), ("fail", ctypes.c_int),
                ("status", ctypes.c_int), ("pass_active", ctypes.c_int),
                ("S1", _D4), ("S2", _D4), ("W", _D4), ("mean", _D4), ("M2", _D4), ("sumI", _D4),
                ("zero", ctypes.c_int * cg.MAX_COMP), ("integral", _D4), ("error", _D4), ("chi2", _D4),
                ("prob", _D4)]


NDIM, NBINS, NSTART, NINC, MAXEVAL = 3, 16, 1000, 500, 20000


def _spec():
    g = cg.genz(NDIM, [cg.GAUSSIAN, cg.C0], np.full((2, NDIM), 1.0), np.full((2, NDIM), 0.4))
    return cg.spec(g, nbins=NBINS, flags=cg.JIT, epsrel=1e-3, maxeval=MAXEVAL, nstart=NSTART, nincrease=NINC,
                   seed=7)


def _header(sp):
    h = Header()
    h.magic = b"CUBAGPU"
    h.version = 2
    h.state_bytes = ctypes.sizeof(State)
    h.ndim, h.ncomp, h.nbins = sp.g.ndim, sp.g.ncomp, sp.nbins
    h.flags = sp.flags & (cg.FP64 | cg.JIT | cg.SCRAMBLE | cg.PSEUDO)
    for c in range(sp.g.ncomp):
        h.family[c] = sp.g.family[c]
        for d in range(sp.g.ndim):
            h.a[c][d], h.u[c][d] = sp.g.a[c][d], sp.g.u[c][d]
    h.epsrel, h.epsabs = sp.epsrel, sp.epsabs
    h.mineval, h.maxeval, h.nstart, h.nincrease, h.seed = sp.mineval, sp.maxeval, sp.nstart, sp.nincrease, sp.seed
    return h


def _state(iters, stopped=False):
    s = State()
    sizes = [NSTART + j * NINC for j in range(iters)]
    s.iter, s.neval, s.stopped = iters, sum(sizes), int(stopped)
    if stopped:
        s.n_cur, s.next_index = sizes[-1], 1 + sum(sizes[:-1])
    else:
        s.n_cur, s.next_index = NSTART + iters * NINC, 1 + sum(sizes)
    return s


def _write(path, header, state, edges=None, H=None, tail=b""):
    edges = np.tile(np.linspace(0.0, 1.0, NBINS + 1), (NDIM, 1)) if edges is None else edges
    H = np.zeros((NDIM, NBINS)) if H is None else H
    with open(path, "wb") as f:
        f.write(bytes(header))
        f.write(bytes(state))
        f.write(np.ascontiguousarray(edges, dtype=np.float64).tobytes())
        f.write(np.ascontiguousarray(H, dtype=np.float64).tobytes())
        f.write(np.zeros(2 * LOG_CAP * cg.MAX_COMP).tobytes())
        f.write(tail)


@pytest.fixture(scope="module")
def lib():
    cg.build_library()
    return cg.lib()


def _jmax():
    j, total = 0, 0
    while total + NSTART + j * NINC <= MAXEVAL:
        total += NSTART + j * NINC
        j += 1
    return j


@pytest.mark.parametrize("iters,stopped", [(0, False), (3, False), (3, True), (_jmax(), True)])
def test_well_formed_state_is_accepted(lib, tmp_path, iters, stopped):
    sp = _spec()
    path = str(tmp_path / "s.bin")
    _write(path, _header(sp), _state(iters, stopped))
    assert cg.check_state_file(sp, path) == (True, "")


def _damage(kind):
    sp = _spec()
    h, s = _header(sp), _state(3)
    edges = np.tile(np.linspace(0.0, 1.0, NBINS + 1), (NDIM, 1))
    H = np.zeros((NDIM, NBINS))
    tail = b""
    if kind == "other problem":
        h.a[0][1] = 1.5
    elif kind == "other format":
        h.version = 1
    elif kind == "edges not increasing":
        edges[1, 5], edges[1, 6] = edges[1, 6], edges[1, 5]
    elif kind == "edges end below 1":
        edges[2, -1] = 0.999
    elif kind == "edges NaN":
        edges[0, 3] = np.nan
    elif kind == "histogram negative":
        H[1, 2] = -1e-30
    elif kind == "histogram infinite":
        H[0, 0] = np.inf
    elif kind == "iteration negative":
        s.iter = -1
    elif kind == "iterations beyond schedule":
        s.iter = _jmax() + 1
    elif kind == "neval off":
        s.neval += 1
    elif kind == "n_cur off":
        s.n_cur += NINC
    elif kind == "next index off":
        s.next_index += 1
    elif kind == "next index past the limit":
        s.next_index = cg.INDEX_LIMIT
    elif kind == "stopped flag":
        s.stopped = 2
    elif kind == "status bits":
        s.status = 4
    elif kind == "trailing bytes":
        tail = b"\0"
    return sp, h, s, edges, H, tail


REASONS = {
    "other problem": "another problem", "other format": "another problem or format",
    "edges not increasing": "not increasing", "edges end below 1": "from 0 to 1", "edges NaN": "not increasing",
    "histogram negative": "histogram", "histogram infinite": "histogram",
    "iteration negative": "iteration count", "iterations beyond schedule": "iteration count",
    "neval off": "sample count", "n_cur off": "next iteration's size", "next index off": "Sobol index",
    "next index past the limit": "Sobol index", "stopped flag": "flags", "status bits": "flags",
    "trailing bytes": "bytes after",
}


@pytest.mark.parametrize("kind", sorted(REASONS))
def test_damaged_state_is_refused_with_its_reason(lib, tmp_path, kind):
    sp, h, s, edges, H, tail = _damage(kind)
    path = str(tmp_path / "s.bin")
    _write(path, h, s, edges, H, tail)
    ok, why = cg.check_state_file(sp, path)
    assert not ok and REASONS[kind] in why, (kind, why)


@pytest.mark.parametrize("cut", [1, 100, 3000, -8])
def test_truncated_state_is_refused(lib, tmp_path, cut):
    sp = _spec()
    full = str(tmp_path / "full.bin")
    _write(full, _header(sp), _state(2))
    data = open(full, "rb").read()
    path = str(tmp_path / "cut.bin")
    open(path, "wb").write(data[:cut] if cut > 0 else data[:len(data) + cut])
    ok, why = cg.check_state_file(sp, path)
    assert not ok and ("truncated" in why or "another problem" in why), why


def test_missing_file_and_bad_spec(lib, tmp_path):
    sp = _spec()
    ok, why = cg.check_state_file(sp, str(tmp_path / "none.bin"))
    assert not ok and "cannot open" in why
    bad = _spec()
    bad.nbins = 1
    path = str(tmp_path / "s.bin")
    _write(path, _header(sp), _state(0))
    ok, why = cg.check_state_file(bad, path)
    assert not ok and "nbins" in why
