"""CPU checks of the C ABI boundary: the library builds, loads and exports every
function include/gpsparse.h declares; host-only calls behave.  No GPU needed."""

import ctypes
import os
import re

import pytest

from paper_2205_09070_gb300 import build as B
from paper_2205_09070_gb300 import gpsparse as G

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "gpsparse.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|void|const char\*)\s+(gp_\w+)\s*\(", text, re.M)))


def test_library_builds_and_exports_header_symbols():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(G.EXPORTED)


def test_host_only_calls():
    G.load()
    d = G.KernelDesc(3, 4, 8, 1.0)
    assert G.load().gp_n_params(ctypes.byref(d)) == 163
    d = G.KernelDesc(2, 2, 3, 1.0)
    assert G.load().gp_n_params(ctypes.byref(d)) == 27
    o = G.default_opts()
    assert o.precision == G.GP_FP32_MIXED and o.n_probes == 32 and o.lanczos_steps == 50
    assert o.cg_rtol == pytest.approx(1e-6)
    assert o.precond_block == 128
    for s in range(9):
        assert G.status_string(s)
    assert G.status_string(G.GP_ERR_NOT_SPD).startswith("CG breakdown")


def test_create_rejects_bad_descriptors_before_touching_a_device():
    lib = G.load()
    h = ctypes.c_void_p()
    for bad in [G.KernelDesc(0, 1, 1, 1.0), G.KernelDesc(2, 0, 1, 1.0), G.KernelDesc(2, 1, 1, -1.0)]:
        assert lib.gp_create(ctypes.byref(h), ctypes.byref(bad), 0, None) == G.GP_ERR_INVALID_ARG
    for big in [G.KernelDesc(4, 1, 1, 1.0), G.KernelDesc(2, 33, 1, 1.0), G.KernelDesc(2, 32, 17, 1.0)]:
        assert lib.gp_create(ctypes.byref(h), ctypes.byref(big), 0, None) == G.GP_ERR_UNSUPPORTED


def test_header_constants_and_info_layout_match_the_binding():
    text = open(HEADER).read()
    defines = dict(re.findall(r"^#define\s+(GP_\w+)\s+(\d+)\b", text, re.M))
    for name, value in defines.items():
        if hasattr(G, name):
            assert getattr(G, name) == int(value), name
    for name in ("GP_FLAG_SPMM_CPASYNC", "GP_FLAG_SPMM_TMA", "GP_FLAG_SPMM_TMA_WIDE", "GP_SPMM_CPASYNC",
                 "GP_SPMM_TMA", "GP_SPMM_TMA_WIDE"):
        assert name in defines and hasattr(G, name), name
    # gp_info's members in declaration order equal the ctypes mirror's fields
    body = text[text.index("typedef struct {\n  int64_t n;"):text.index("} gp_info;")]
    members = re.findall(r"^\s*(?:int64_t|int32_t|double)\s+(\w+);", body, re.M)
    assert members == [f for f, _ in G.Info._fields_]


def test_header_is_plain_c():
    # the boundary is a C ABI: the header must compile as C99 on its own
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    r = subprocess.run([cc, "-x", "c", "-std=c99", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", HEADER],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
