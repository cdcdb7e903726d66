"""The binding's ctypes structures lay out exactly as the C header's
structs: every struct's size and every field's offset, from a small C
program compiled against include/cubagpu.h with the host compiler (no GPU,
no CUDA), so header and binding cannot drift apart unnoticed."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_1408_6373_gb300 as cg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "cv_genz": cg.Genz,
    "cv_spec": cg.Spec,
    "cv_result": cg.Result,
    "cv_server_opts": cg.ServerOpts,
    "cv_serve_stats": cg.ServeStats,
    "cv_genz_cb_data": cg.GenzCallbackData,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("layout")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "cubagpu.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, value = line.split()
        layout[(name, field)] = int(value)
    return layout


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_struct_layout_matches_header(c_layout, cname):
    py = STRUCTS[cname]
    assert ctypes.sizeof(py) == c_layout[(cname, "size")], cname
    for fname, _ in py._fields_:
        assert getattr(py, fname).offset == c_layout[(cname, fname)], (cname, fname)


def test_binding_constants_match_header_macros():
    # the integer macros of the header, evaluated by the C preprocessor's
    # own arithmetic through the host compiler, against the binding's names
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    pairs = {"CV_MAX_DIM": cg.MAX_DIM, "CV_MAX_COMP": cg.MAX_COMP, "CV_MIN_BINS": cg.MIN_BINS,
             "CV_MAX_BINS": cg.MAX_BINS, "CV_INDEX_LIMIT": cg.INDEX_LIMIT, "CV_TIMER_CAP": cg.KERNEL_TIMER_CAP,
             "CV_STATIC_SCRATCH_BYTES": cg.STATIC_SCRATCH_BYTES, "CV_OK": cg.OK, "CV_EINVAL": cg.EINVAL,
             "CV_ENOMEM": cg.ENOMEM, "CV_ECUDA": cg.ECUDA, "CV_EABORT": cg.EABORT, "CV_ETIMEOUT": cg.ETIMEOUT,
             "CV_EADMIT": cg.EADMIT, "CV_EBUSY": cg.EBUSY, "CV_ENOTFOUND": cg.ENOTFOUND,
             "CV_ESCRATCH": cg.ESCRATCH, "CV_ENONFINITE": cg.ENONFINITE, "CV_FP64": cg.FP64,
             "CV_PLAIN": cg.PLAIN, "CV_AOS": cg.AOS, "CV_JIT": cg.JIT, "CV_SCRAMBLE": cg.SCRAMBLE,
             "CV_PSEUDO": cg.PSEUDO, "CV_CORNER_PEAK": cg.CORNER_PEAK, "CV_CONST": cg.CONST}
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        lines = ["#include <stdio.h>", '#include "cubagpu.h"', "int main(void) {"]
        lines += [f'    printf("{k} %lld\\n", (long long)({k}));' for k in pairs]
        lines += ["    return 0;", "}"]
        src = os.path.join(d, "c.c")
        open(src, "w").write("\n".join(lines) + "\n")
        exe = os.path.join(d, "c")
        subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    got = {k: int(v) for k, v in (line.split() for line in out.splitlines())}
    assert got == pairs
