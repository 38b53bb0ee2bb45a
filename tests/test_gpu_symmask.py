"""The direct operators for a mirror-symmetric mask with the mask factor computed
online (CAXSI_OPT_ONLINE_MASK): parity with the FP64 oracle, agreement with the
per-pair-bit kernels, the adjoint identity, and the refusal for masks without
the symmetry."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def cx():
    import torch
    from paper_1603_06400_gb300 import build, caxsi
    build.build()
    return caxsi, torch


def _t(torch, a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda:0")


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


GEOMS = {
    "tiny": lambda: synth.tiny_geometry(),
    # ragged quadrant tiles (M/2 = 5 rows, N/2 = 20 columns) and odd rho_y
    "ragged": lambda: synth.make_geometry(X=5, J=6, Q=24, M=10, N=40, K=12, rho_y=3, p_y=194.56 / 40,
                                          p_z=2 * 194.56 / 40, dx=14.0),
    # many voxels per detector row: adjoint rows in one range, forward chunks of pairs
    "wide": lambda: synth.make_geometry(X=8, J=64, Q=16, M=4, N=64, K=8, rho_y=1, p_y=3.04, p_z=6.08,
                                        dx=8.75),
}


@pytest.mark.parametrize("name", sorted(GEOMS))
def test_online_symmetric_mask_operators(cx, name):
    caxsi, torch = cx
    g = GEOMS[name]()
    phi = synth.tungsten_spectrum(g)
    mask = synth.symmetric_mask(g, 77)
    plan = caxsi.Plan(g, phi, mask)
    assert plan.info()["mask_symmetric"] == 1
    f = synth.phantom(g, 5, n_ellipses=3) + 0.05 * synth.uniform_random((g.X, g.J, g.Q), 1)
    w = synth.uniform_random((g.M, g.N), 2) + 0.1
    D = caxsi.PATH_DIRECT
    g_bits = plan.forward(_t(torch, f), path=D).double().cpu().numpy()
    f_bits = plan.adjoint(_t(torch, w), path=D).double().cpu().numpy()
    plan.set_online_mask(True)
    g_on = plan.forward(_t(torch, f), path=D).double().cpu().numpy()
    f_on = plan.adjoint(_t(torch, w), path=D).double().cpu().numpy()
    ref_g = oracle.forward(g, phi, mask, _f32(f))
    ref_f = oracle.adjoint(g, phi, mask, _f32(w))
    assert rel_l2(g_on, ref_g) <= 1e-5 and rel_l2(f_on, ref_f) <= 1e-5
    # the same per-pair values as the per-pair-bit kernels, summed in another order
    assert rel_l2(g_on, g_bits) <= 2e-6 and rel_l2(f_on, f_bits) <= 2e-6
    # the forward image is up-down symmetric by construction (f has no z dependence)
    np.testing.assert_array_equal(g_on, g_on[::-1, :])
    # adjoint identity with FP64 dot products
    lhs = float(np.sum(g_on * w))
    rhs = float(np.sum(_f32(f) * f_on))
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)
    # deterministic
    assert np.array_equal(plan.forward(_t(torch, f), path=D).double().cpu().numpy(), g_on)
    plan.set_online_mask(False)
    assert np.array_equal(plan.forward(_t(torch, f), path=D).double().cpu().numpy(), g_bits)
    plan.close()


def test_online_mask_needs_a_symmetric_mask(cx, tiny):
    caxsi, torch = cx
    g, phi, mask = tiny
    plan = caxsi.Plan(g, phi, mask)            # a random mask: no mirror symmetry
    assert plan.info()["mask_symmetric"] == 0
    with pytest.raises(caxsi.CaxsiError) as e:
        plan.set_online_mask(True)
    assert e.value.status == 6
    plan.close()
    # a symmetric pattern on a grid that is not centred on the central ray
    gs = g.with_(mask_y0=g.mask_y0 + 0.5 * g.mask_cell)
    plan = caxsi.Plan(gs, phi, synth.symmetric_mask(g, 3))
    assert plan.info()["mask_symmetric"] == 0
    plan.close()
    # odd detector rows: the up-down images are not pixels
    go = synth.make_geometry(X=4, J=6, Q=16, M=9, N=40, K=8, rho_y=2, p_y=4.864, p_z=9.728, dx=14.0)
    plan = caxsi.Plan(go, synth.tungsten_spectrum(go), synth.symmetric_mask(go, 4))
    assert plan.info()["mask_symmetric"] == 0
    plan.close()


def test_paper_scale_symmetric_mask_sampled(cx):
    caxsi, torch = cx
    g = synth.paper_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.symmetric_mask(g, 1003)
    plan = caxsi.Plan(g, phi, mask)
    plan.set_online_mask(True)
    f = synth.phantom(g, 0)
    w = synth.uniform_random((g.M, g.N), 1) + 0.5
    D = caxsi.PATH_DIRECT
    gg = plan.forward(_t(torch, f), path=D).cpu().numpy().ravel()
    fa = plan.adjoint(_t(torch, w), path=D).cpu().numpy().reshape(g.X * g.J, g.Q)
    rng = np.random.default_rng(5)
    pix = np.concatenate([rng.choice(g.M * g.N, 40, replace=False), [0, g.M * g.N - 1]])
    assert rel_l2(gg[pix], oracle.forward_pixels(g, phi, mask, _f32(f), pix)) <= 1e-5
    vox = np.concatenate([rng.choice(g.X * g.J, 24, replace=False), [0, g.X * g.J - 1]])
    assert rel_l2(fa[vox], oracle.adjoint_voxels(g, phi, mask, _f32(w), vox)) <= 1e-5
    plan.close()
