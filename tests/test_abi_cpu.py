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
