"""Host-side checks of the C ABI: the library builds, loads, exports every
function include/qmlgb.h declares, and rejects bad arguments before touching
the GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2605_21149_gb300 import _native as nat
from paper_2605_21149_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return nat.load()


def test_every_declared_symbol_is_exported(lib):
    decl = header_functions()
    assert {"qml_fisher", "qml_estimate", "pix_loglike", "qml_ybuild"} <= decl
    for name in decl:
        assert hasattr(lib, name), name
    assert decl == set(nat.SIGNATURES), decl ^ set(nat.SIGNATURES)


def test_version_and_error_string(lib):
    assert lib.qml_version() >= 100
    assert isinstance(lib.qml_last_error(), bytes)


def _problem(**kw):
    p = nat.QmlProblem()
    p.has_T, p.has_P = 1, 0
    p.npix_T = 10
    buf = (ctypes.c_double * 64)()
    ptr = ctypes.cast(buf, ctypes.c_void_p)
    p.theta_T = p.phi_T = p.transfer_T = ptr
    p.lmin, p.lmax = 2, 5
    p.nspec = 1
    p.spec[0] = 0
    p.cl_fid = ptr
    p.N = ptr
    for k, v in kw.items():
        setattr(p, k, v)
    return p, buf


@pytest.mark.parametrize("field,value,needle", [
    ("lmin", 1, "lmin"),
    ("lmax", 1, "lmax"),
    ("nspec", 0, "nspec"),
    ("has_T", 0, "no field"),
    ("npix_T", 0, "npix_T"),
    ("precision", 7, "precision"),
])
def test_argument_validation(lib, field, value, needle):
    p, keep = _problem(**{field: value})
    F = (ctypes.c_double * 16)()
    st = lib.qml_fisher(ctypes.byref(p), ctypes.cast(F, ctypes.c_void_p), None, None)
    assert st == nat.QML_EINVAL
    assert needle in lib.qml_last_error().decode()


def test_spectrum_needs_its_field(lib):
    p, keep = _problem()
    p.spec[0] = 1  # EE without a polarisation field
    F = (ctypes.c_double * 16)()
    assert lib.qml_fisher(ctypes.byref(p), ctypes.cast(F, ctypes.c_void_p), None, None) == nat.QML_EINVAL
    assert "absent" in lib.qml_last_error().decode()


def test_null_problem(lib):
    assert lib.qml_ybuild(None, None, 0, None) == nat.QML_EINVAL
    assert lib.qml_estimate(None, None, 0, None, None, None, None, None, None) == nat.QML_EINVAL
    assert lib.qml_potrf(0, None, 0, None, 0, None) == nat.QML_EINVAL


def test_tuning_table_round_trip(lib):
    """The tuning table (qml_tune_*) is host state: set, get, dump, reload."""
    from paper_2605_21149_gb300 import api
    api.tune_set("test_key_alpha", 17)
    assert api.tune_get("test_key_alpha") == 17
    assert api.tune_get("no_such_key_for_sure") is None
    text = api.tune_table()
    assert "test_key_alpha 17\n" in text
    api.tune_set("test_key_alpha", 3)
    api.tune_load("# comment\ntest_key_alpha 17\ntest_key_beta -5\n")
    assert api.tune_get("test_key_alpha") == 17 and api.tune_get("test_key_beta") == -5
    # malformed text is rejected and leaves the table unchanged
    assert lib.qml_tune_load(b"test_key_alpha 1\nbroken line here\n") != 0
    assert api.tune_get("test_key_alpha") == 17
    assert lib.qml_tune_set(b"bad key", 1) != 0
    # a too-small buffer is left untouched and the needed size returned
    need = lib.qml_tune_table(None, 0)
    buf = ctypes.create_string_buffer(b"x" * 4)
    assert lib.qml_tune_table(buf, 4) == need and buf.raw[:4] == b"xxxx"


def _bins(edges):
    arr = (ctypes.c_int32 * len(edges))(*edges)
    return len(edges) - 1, ctypes.cast(arr, ctypes.c_void_p), arr


@pytest.mark.parametrize("edges,needle", [
    ([3, 4, 6], "lmin"),          # must start at lmin = 2
    ([2, 4, 5], "lmax + 1"),      # must end at lmax + 1 = 6
    ([2, 4, 4, 6], "increase"),
    ([2, 3, 4, 5, 6, 7], "more bins"),
])
def test_bin_edge_validation(lib, edges, needle):
    """Native binning (Sect. 2.4): qml_fisher rejects bad edges before any
    device work."""
    nb, ptr, keep_edges = _bins(edges)
    p, keep = _problem(nbins=nb, bin_edges=ptr)
    F = (ctypes.c_double * 64)()
    assert lib.qml_fisher(ctypes.byref(p), ctypes.cast(F, ctypes.c_void_p), None, None) == nat.QML_EINVAL
    assert needle in lib.qml_last_error().decode()


def test_bin_edges_null_and_negative(lib):
    F = (ctypes.c_double * 64)()
    p, keep = _problem(nbins=2, bin_edges=None)
    assert lib.qml_fisher(ctypes.byref(p), ctypes.cast(F, ctypes.c_void_p), None, None) == nat.QML_EINVAL
    p, keep = _problem(nbins=-1)
    assert lib.qml_fisher(ctypes.byref(p), ctypes.cast(F, ctypes.c_void_p), None, None) == nat.QML_EINVAL


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of qml_problem and lnl_mask have the C layout
    (sizes and field offsets from the header, compiled with gcc)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    fields = [f[0] for f in nat.QmlProblem._fields_]
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "qmlgb.h"\nint main(void) {\n'
                   '  printf("%zu %zu\\n", sizeof(qml_problem), sizeof(lnl_mask));\n' +
                   "".join(f'  printf("%zu\\n", offsetof(qml_problem, {f}));\n' for f in fields) +
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(nat.QmlProblem)
    assert int(out[1]) == ctypes.sizeof(nat.LnlMask)
    for f, off in zip(fields, out[2:]):
        assert int(off) == getattr(nat.QmlProblem, f).offset, f
