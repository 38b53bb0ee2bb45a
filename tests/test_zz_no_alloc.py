"""The forward entry point whose scratch is a static device array.

caxsi_forward_static_scratch serves callers that must not allocate device
memory when they call it (code running while another thread captures a CUDA
graph in global mode, real-time loops that forbid allocation after start-up,
hosts whose memory pool owns the device).  It is checked here, through the C
ABI, against the plan-scratch forward on two calls in a row, and its size
limit is checked to be refused before anything runs.  This file is collected
last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

REL_L2_TOL = 1e-5
SCRATCH_FLOATS = 1 << 20   # CAXSI_STATIC_SCRATCH_FLOATS in include/caxsi.h


def _rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_static_scratch_forward_matches_plan_forward():
    import torch
    from paper_1603_06400_gb300 import build, caxsi
    build.build()
    lib = caxsi.load()
    for g in (synth.tiny_geometry(), synth.paper_geometry()):
        phi = synth.tungsten_spectrum(g)
        mask = synth.random_mask(g, 1234)
        plan = caxsi.Plan(g, phi, mask)
        f = torch.tensor(synth.phantom(g, 4, n_ellipses=3), dtype=torch.float32, device="cuda:0")
        ref = plan.forward(f, path=caxsi.PATH_DIRECT).cpu().numpy()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        out = torch.empty((g.M, g.N), dtype=torch.float32, device="cuda:0")
        outs = []
        for call in range(2):
            out.fill_(float("nan"))
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            st = lib.caxsi_forward_static_scratch(plan.handle, ctypes.c_void_p(f.data_ptr()),
                                                  g.f_len, ctypes.c_void_p(out.data_ptr()),
                                                  g.g_len, stream)
            assert st == 0, lib.caxsi_status_string(st)
            torch.cuda.synchronize()
            if call == 1:   # the first call may look up the array's address; later ones never allocate
                assert torch.cuda.mem_get_info()[0] == free_before
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert _rel_l2(got, ref) <= REL_L2_TOL
            outs.append(got)
        np.testing.assert_array_equal(outs[0], outs[1])
        plan.close()


def test_static_scratch_rejects_oversize_detector():
    import torch
    from paper_1603_06400_gb300 import build, caxsi
    build.build()
    lib = caxsi.load()
    g = synth.make_geometry(X=1, J=1, Q=2, M=1025, N=1024, K=1, rho_y=1, p_y=0.1, p_z=0.1,
                            dx=1.0, mask_cell=5.0)
    assert g.M * g.N > SCRATCH_FLOATS
    plan = caxsi.Plan(g, synth.tungsten_spectrum(g), synth.random_mask(g, 5))
    f = torch.ones(g.f_len, dtype=torch.float32, device="cuda:0")
    out = torch.zeros(g.g_len, dtype=torch.float32, device="cuda:0")
    st = lib.caxsi_forward_static_scratch(plan.handle, ctypes.c_void_p(f.data_ptr()), g.f_len,
                                          ctypes.c_void_p(out.data_ptr()), g.g_len, None)
    assert st == 7
    assert lib.caxsi_status_string(st).decode() == "problem exceeds the static scratch array"
    assert lib.caxsi_forward_static_scratch(plan.handle, None, g.f_len, None, g.g_len, None) == 1
    plan.close()
