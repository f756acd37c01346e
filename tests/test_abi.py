"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/srt.h, and validates arguments before any CUDA call."""
import ctypes
import math
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "srt.h")


@pytest.fixture(scope="module")
def L():
    from paper_2402_15641_gb300 import build, _lib
    build.build()
    return _lib


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(srt_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("srt_plan", "srt_forward", "srt_adjoint", "srt_plan_destroy", "srt_plan_info",
                 "srt_workspace_bytes", "srt_error_string", "srt_dot_f64"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (srt_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = L.lib()
    for n in declared_functions():
        assert hasattr(lib, n)
        assert n in L.SIGNATURES, f"{n} has no ctypes signature"


def test_struct_layout_matches_header(L, tmp_path):
    """ctypes mirrors agree with the C compiler's sizeof/offsetof for the header."""
    fields = {"srt_geometry": L.SrtGeometry, "srt_plan_info_t": L.SrtPlanInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "srt.h"', "int main(void){"]
    for cname, py in fields.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n"):
        if ln:
            a, b, c = ln.split()
            got[(a, b)] = int(c)
    for cname, py in fields.items():
        assert got[(cname, "size")] == ctypes.sizeof(py)
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_error_strings(L):
    lib = L.lib()
    for code in range(8):
        s = lib.srt_error_string(code).decode()
        assert s and s != "unknown status"
    assert lib.srt_error_string(99).decode() == "unknown status"


def test_geometry_default_readings(L):
    g = L.SrtGeometry()
    assert L.lib().srt_geometry_default(ctypes.byref(g), 32, 32, 0.5, 0.5, 12.0, 64, 32, 96) == 0
    rxy = 32 * 0.5 / math.sqrt(2)
    assert g.ell_lo == pytest.approx(12 - rxy, abs=1e-15)
    assert g.ell_hi == pytest.approx(12 + rxy, abs=1e-15)
    assert (g.zs_lo, g.zs_hi, g.phi0, g.weight_dtype, g.flags) == (-8.0, 8.0, 0.0, 0, 0)
    assert L.lib().srt_geometry_default(None, 1, 1, 1, 1, 1, 1, 1, 1) == L.SRT_ERR_ARG


def test_geometry_matches_oracle_default(L, orc):
    from paper_2402_15641_gb300.srt import Geometry
    for sz in [(32, 32, 0.5, 0.5, 12.0, 64, 32, 96), (256, 256, 0.1, 0.1, 20.0, 256, 256, 768)]:
        a = Geometry.default(*sz)
        b = orc.OracleGeometry.default(*sz)
        for k in ("ms", "mz", "dxy", "dz", "radius", "n_phi", "phi0", "n_zs", "zs_lo", "zs_hi",
                  "n_ell", "ell_lo", "ell_hi"):
            assert getattr(a, k) == getattr(b, k), k


def _plan_status(L, **kw):
    g = L.SrtGeometry()
    L.lib().srt_geometry_default(ctypes.byref(g), 8, 8, 0.5, 0.5, 5.0, 8, 8, 16)
    for k, v in kw.items():
        setattr(g, k, v)
    h = ctypes.c_void_p(123)
    s = L.lib().srt_plan(ctypes.byref(g), None, ctypes.byref(h))
    return s, h.value


@pytest.mark.parametrize("kw", [dict(ms=0), dict(mz=-1), dict(n_phi=0), dict(n_ell=0),
                                dict(dxy=0.0), dict(dz=-1.0), dict(radius=2.0),
                                dict(ell_lo=0.0), dict(ell_lo=-1.0), dict(ell_hi=1.0),
                                dict(zs_hi=-10.0), dict(weight_dtype=7), dict(phi0=float("nan")),
                                # index ranges beyond int32: pixels, A1 rows, (radius, slab) cells
                                dict(ms=46341, radius=1e6), dict(n_phi=1 << 20, n_ell=1 << 12),
                                dict(mz=1 << 20, n_ell=1 << 12)])
def test_invalid_geometry_rejected_before_device_work(L, kw):
    s, h = _plan_status(L, **kw)
    assert s == L.SRT_ERR_GEOMETRY
    assert h is None


def test_null_arguments(L):
    lib = L.lib()
    h = ctypes.c_void_p()
    assert lib.srt_plan(None, None, ctypes.byref(h)) == L.SRT_ERR_ARG
    assert lib.srt_plan(None, None, None) == L.SRT_ERR_ARG
    assert lib.srt_forward(None, None, None, 1, None, 0, None) == L.SRT_ERR_ARG
    assert lib.srt_adjoint(None, None, None, 1, None, 0, None) == L.SRT_ERR_ARG
    n = ctypes.c_size_t()
    assert lib.srt_workspace_bytes(None, 1, ctypes.byref(n)) == L.SRT_ERR_ARG
    assert lib.srt_plan_info(None, None) == L.SRT_ERR_ARG
    assert lib.srt_plan_destroy(None) == 0
    assert lib.srt_dot_workspace_bytes() >= 8
    assert lib.srt_dot_f64(None, None, 1, None, None, 0, None) == L.SRT_ERR_ARG
    q = ctypes.c_void_p(1)
    assert lib.srt_pipe_create(None, 1, 2, ctypes.byref(q)) == L.SRT_ERR_ARG and not q.value
    assert lib.srt_pipe_create(None, 1, 2, None) == L.SRT_ERR_ARG
    tk = ctypes.c_int64()
    assert lib.srt_pipe_submit(None, 0, None, None, ctypes.byref(tk)) == L.SRT_ERR_ARG
    assert lib.srt_pipe_wait(None, 0, 1.0) == L.SRT_ERR_ARG
    assert lib.srt_pipe_destroy(None) == 0


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2402_15641_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.lib()



@pytest.mark.parametrize("compiler,std,ext", [("gcc", "-std=c99", "c"), ("g++", "-std=c++11", "cpp")])
def test_header_is_strict_c99_and_cxx11(tmp_path, compiler, std, ext):
    """The boundary header compiles warning-free as C99 and as C++11 (its
    extern "C" block), with -Wall -Wextra -pedantic -Werror."""
    src = tmp_path / f"probe.{ext}"
    src.write_text('#include "srt.h"\n'
                   "int main(void) { srt_geometry g; srt_plan_info_t i; (void)g; (void)i;\n"
                   "  return SRT_OK; }\n")
    subprocess.run([compiler, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                    os.path.join(ROOT, "include"), "-fsyntax-only", str(src)], check=True)
