"""The C ABI library loads and exports what include/caxsi.h declares; argument
validation answers without touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1603_06400_gb300 import build as B
from paper_1603_06400_gb300 import caxsi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return caxsi.load()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(caxsi_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("caxsi_plan_create", "caxsi_plan_destroy", "caxsi_forward", "caxsi_adjoint",
                 "caxsi_recon_step", "caxsi_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code, text in caxsi.STATUS.items():
        assert lib.caxsi_status_string(code).decode()
    assert lib.caxsi_status_string(99).decode() == "unknown status"


def test_null_and_invalid_arguments_rejected_before_any_cuda_call(lib):
    import synth
    g = synth.tiny_geometry()
    P = ctypes.c_void_p
    out = P()
    phi = np.ones(g.K)
    mask = np.ones((g.mask_rows, g.mask_cols), np.uint8)
    dp = phi.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    mp = mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    gs = caxsi.geometry_struct(g)
    assert lib.caxsi_plan_create(None, dp, mp, ctypes.byref(out)) == 1
    assert lib.caxsi_plan_create(ctypes.byref(gs), None, mp, ctypes.byref(out)) == 1
    assert lib.caxsi_plan_create(ctypes.byref(gs), dp, None, ctypes.byref(out)) == 1
    assert lib.caxsi_plan_create(ctypes.byref(gs), dp, mp, None) == 1
    for bad in (dict(Q=1), dict(X=0), dict(K=0), dict(rho_y=0), dict(p_y=-1.0), dict(dx=0.0),
                dict(q_max=0.05), dict(E_min=-1.0), dict(X_mask=2000.0), dict(x_center=-5.0),
                dict(hc=float("nan")), dict(K=5000), dict(mask_cols=0)):
        bg = caxsi.geometry_struct(g.with_(**bad))
        assert lib.caxsi_plan_create(ctypes.byref(bg), dp, mp, ctypes.byref(out)) == 1, bad
    nan_phi = phi.copy()
    nan_phi[3] = np.nan
    assert lib.caxsi_plan_create(ctypes.byref(gs), nan_phi.ctypes.data_as(
        ctypes.POINTER(ctypes.c_double)), mp, ctypes.byref(out)) == 1
    assert out.value is None
    # calls on a null plan
    assert lib.caxsi_forward(None, None, 0, None, 0, 0, None) == 1
    assert lib.caxsi_adjoint(None, None, 0, None, 0, 0, None) == 1
    assert lib.caxsi_recon_step(None, None, None, None, 0, 0.0, 0.0, 0, None, None) == 1
    assert lib.caxsi_forward_host(None, None, 0, None, 0, 0) == 1
    info = caxsi.CPlanInfo()
    assert lib.caxsi_plan_info(None, ctypes.byref(info)) == 1
    sub = np.zeros(g.M * g.N, np.int32)
    assert lib.caxsi_plan_set_subsets(None, 1, sub.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))) == 1
    assert lib.caxsi_forward_subset(None, 0, None, 0, None, 0, 1, None) == 1
    assert lib.caxsi_adjoint_subset(None, 0, None, 0, None, 0, 1, None) == 1
    assert lib.caxsi_recon_step_subset(None, 0, None, None, None, 0, 0.0, 0.0, 1, None, None) == 1
    lib.caxsi_plan_destroy(None)


# --------------------------------------------------------------------------
# The binding agrees with the headers: struct layouts (compiled by gcc from the
# header itself) and the parameter list of every declared function
# --------------------------------------------------------------------------

def _strip_comments(txt):
    txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
    return re.sub(r"//[^\n]*", " ", txt)


def _declarations():
    """name -> parameter kinds ('ptr', 'i32', 'i64', 'f32', 'f64') of every
    function declared in include/*.h."""
    kinds = {"int": "i32", "int32_t": "i32", "caxsi_status": "i32", "int64_t": "i64", "uint64_t": "i64",
             "float": "f32", "double": "f64"}
    out = {}
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = _strip_comments(open(os.path.join(ROOT, "include", h)).read())
        for name, params in re.findall(r"\b(caxsi_\w+)\s*\(([^;{}()]*)\)\s*;", txt):
            ps = [p.strip() for p in params.split(",") if p.strip()]
            if ps == ["void"]:
                ps = []
            ks = []
            for p in ps:
                if "*" in p:
                    ks.append("ptr")
                    continue
                words = p.replace("const", " ").split()
                assert len(words) == 2, (name, p)       # type and parameter name
                ks.append(kinds[words[0]])
            out[name] = ks
    return out


def _kind(ct):
    if ct in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(ct, type) and issubclass(ct, ctypes._Pointer)):
        return "ptr"
    sizes = {ctypes.c_int: "i32", ctypes.c_int32: "i32", ctypes.c_int64: "i64", ctypes.c_long: "i64",
             ctypes.c_uint64: "i64", ctypes.c_ulong: "i64",
             ctypes.c_float: "f32", ctypes.c_double: "f64"}
    return sizes[ct]


def test_binding_parameter_lists_match_the_headers(lib):
    decls = _declarations()
    assert len(decls) == len(declared_functions())
    for name, kinds in decls.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, f"{name}: the binding sets no argument types"
        got = [_kind(t) for t in fn.argtypes]
        assert got == kinds, f"{name}: header {kinds}, binding {got}"


def test_struct_layouts_match_the_header(tmp_path):
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"caxsi_geometry": caxsi.CGeometry, "caxsi_plan_info_t": caxsi.CPlanInfo,
               "caxsi_kernel_stat": caxsi.CKernelStat}
    # both public headers compile as plain C11, without CUDA headers
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "caxsi.h"', '#include "caxsi_nn.h"',
             "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, field, value = ln.split()
        got[(cname, field)] = int(value)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert got[(cname, field)] == getattr(cls, field).offset, (cname, field)


def test_binding_return_types_match_the_headers(lib):
    want = {"caxsi_status": ctypes.c_int, "void": None, "const char *": ctypes.c_char_p}
    seen = 0
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = _strip_comments(open(os.path.join(ROOT, "include", h)).read())
        for ret, name in re.findall(r"(caxsi_status|void|const\s+char\s*\*)\s*(caxsi_\w+)\s*\([^;{}()]*\)\s*;", txt):
            ret = "const char *" if "char" in ret else ret
            assert getattr(lib, name).restype is want[ret], (name, ret)
            seen += 1
    assert seen == len(declared_functions())
