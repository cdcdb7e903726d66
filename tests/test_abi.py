"""The C-ABI library loads on the CPU and exports every entry point that
include/cubagpu.h declares (no compute calls: no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1408_6373_gb300 as cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(cv_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    return cg.build_library()


def test_header_declares_entry_points():
    assert {"cv_create", "cv_destroy", "cv_sobol", "cv_sample", "cv_refine", "cv_vegas"} <= _declared()


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in sorted(_declared()):
        assert hasattr(L, name), f"{name} declared but not exported"


def test_binding_covers_every_declared_symbol():
    assert _declared() == set(cg.exported_symbols())


def test_exports_are_plain_c_symbols(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert _declared() <= exported


def test_strerror_without_gpu(libpath):
    L = cg.lib()
    assert L.cv_strerror(-1) == b"invalid argument"
    assert L.cv_strerror(0) == b"ok"


def test_null_context_is_rejected_without_gpu():
    L = cg.lib()
    assert L.cv_sobol(None, 3, 0, 10, 52, None) == cg.EINVAL
    assert L.cv_synchronize(None) == cg.EINVAL


def test_sobol_table_header_is_current(tmp_path):
    # regenerating the direction words reproduces the committed header
    gen = os.path.join(ROOT, "paper_1408_6373_gb300", "csrc", "gen_sobol_dirs.py")
    out = tmp_path / "sobol_dirs.h"
    subprocess.check_call(["python", gen, str(out)], stdout=subprocess.DEVNULL)
    committed = open(os.path.join(ROOT, "paper_1408_6373_gb300", "csrc", "sobol_dirs.h")).read()
    assert out.read_text() == committed
