"""Uniform u-sample tables (CAXSI_OPT_U_SAMPLES): W(r, u) sampled at N uniform u
and interpolated linearly between the samples, the table-path counterpart of the
paper's scatter-angle interpolation (Sec. III-B).

This is an approximation of A, so it is compared with the FP64 oracle by its
error, which must fall as N grows (the interpolation error of a piecewise-linear
W sampled on a uniform grid), and its adjoint must be the exact transpose of the
approximate forward (adjoint identity in FP64 dot products).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def cx():
    import torch
    from paper_1603_06400_gb300 import build, caxsi
    build.build()
    return caxsi, torch


@pytest.fixture(scope="module")
def case():
    g = synth.tiny_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 31)
    f = synth.phantom(g, 4, n_ellipses=3) + 0.05 * synth.uniform_random((g.X, g.J, g.Q), 5)
    w = synth.uniform_random((g.M, g.N), 6) + 0.1
    f64 = np.asarray(f, np.float32).astype(np.float64)
    w64 = np.asarray(w, np.float32).astype(np.float64)
    return g, phi, mask, f, w, oracle.forward(g, phi, mask, f64), oracle.adjoint(g, phi, mask, w64)


def _run(cx, case, n, path="table_fp32"):
    caxsi, torch = cx
    g, phi, mask, f, w, _, _ = case
    plan = caxsi.Plan(g, phi, mask)
    plan.set_u_samples(n)
    P = caxsi.PATHS[path]
    ft = torch.tensor(np.asarray(f, np.float32), device="cuda:0")
    wt = torch.tensor(np.asarray(w, np.float32), device="cuda:0")
    gf = plan.forward(ft, path=P).cpu().numpy().astype(np.float64)
    fa = plan.adjoint(wt, path=P).cpu().numpy().astype(np.float64)
    info = plan.info()
    plan.close()
    return gf, fa, info


def test_error_falls_with_the_number_of_samples(cx, case):
    g, phi, mask, f, w, ref_g, ref_f = case
    errs = []
    for n in (64, 256, 1024, 4096):
        gf, fa, info = _run(cx, case, n)
        assert info["n_breakpoints"] == n
        assert info["device_error"] == 0
        errs.append((rel_l2(gf, ref_g), rel_l2(fa, ref_f)))
    for (a_g, a_f), (b_g, b_f) in zip(errs, errs[1:]):
        assert b_g < a_g and b_f < a_f
    # W is piecewise linear: only the sample intervals that hold one of its kinks
    # err, by O(h) over a length h, so the L2 error falls about as h^1.5 (8x for
    # 4x the samples; 7-8x measured on this case)
    assert errs[-1][0] < 0.25 * errs[-2][0] and errs[-1][1] < 0.25 * errs[-2][1]
    assert errs[-1][0] < 1e-4 and errs[-1][1] < 1e-3


@pytest.mark.parametrize("n", [100, 2048])
def test_adjoint_is_the_transpose_of_the_sampled_forward(cx, case, n):
    g, phi, mask, f, w, _, _ = case
    gf, fa, _ = _run(cx, case, n)
    lhs = float(np.dot(gf.ravel(), np.asarray(w, np.float32).astype(np.float64).ravel()))
    rhs = float(np.dot(np.asarray(f, np.float32).astype(np.float64).ravel(), fa.ravel()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_sampled_table_with_bf16_contractions(cx, case):
    g, phi, mask, f, w, ref_g, ref_f = case
    gf, fa, _ = _run(cx, case, 2048, path="table_bf16")
    g32, f32, _ = _run(cx, case, 2048, path="table_fp32")
    # the bf16 operands add their own rounding (about 4e-5 forward, 2e-4 adjoint
    # with the exact knots) to the sampling error
    assert rel_l2(gf, g32) < 5e-4 and rel_l2(fa, f32) < 1e-3
    assert rel_l2(gf, ref_g) < 2e-4 and rel_l2(fa, ref_f) < 2e-3


def test_option_is_fixed_once_the_table_exists(cx, case):
    caxsi, torch = cx
    g, phi, mask, f, w, _, _ = case
    plan = caxsi.Plan(g, phi, mask)
    plan.set_u_samples(512)
    with pytest.raises(caxsi.CaxsiError):
        plan.set_u_samples(1)            # below 2 and not 0
    with pytest.raises(caxsi.CaxsiError):
        plan.set_u_samples(8193)         # above the maximum
    plan.forward(torch.tensor(np.asarray(f, np.float32), device="cuda:0"), path=caxsi.PATHS["table_fp32"])
    plan.set_u_samples(512)              # unchanged: accepted
    with pytest.raises(caxsi.CaxsiError):
        plan.set_u_samples(0)
    plan.close()
