"""Objects of different geometries in one launch (caxsi_multi_*): every object's
forward model and adjoint against the FP64 oracle, bit-identity with the
single-plan calls, the update and its reverse mode, automatic differentiation
through the packed operator, and 32 objects of uneven size (x across the fan
64-256, z along the beam 32-128, q bins 64-128) on the paper-scale detector.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

REL_L2_TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def cx():
    import torch
    from paper_1603_06400_gb300 import autodiff, build, caxsi
    build.build()
    return caxsi, autodiff, torch


def _t(torch, a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda:0")


def small_objects():
    """Objects small enough for the oracle, of different extents in x, z and q, with
    ragged detector tiles (N not a multiple of 32, M not of 8), different detectors,
    spectra and masks, and both adjoint layouts: tiny objects have their detector
    rows split over several warps (partial rows summed), the 2 560-voxel one not."""
    shapes = [  # X, J, Q, M, N, K, rho_y
        (3, 4, 8, 10, 40, 6, 2),
        (6, 8, 24, 10, 40, 12, 2),
        (2, 5, 37, 6, 20, 9, 4),
        (5, 12, 16, 10, 40, 8, 2),
        (16, 160, 12, 8, 33, 5, 1),
        (1, 1, 64, 12, 70, 16, 2),
    ]
    out = []
    for k, (X, J, Q, M, N, K, rho) in enumerate(shapes):
        py = 194.56 / max(N, J * rho)      # detector and object at most 194.56 mm wide
        g = synth.make_geometry(X=X, J=J, Q=Q, M=M, N=N, K=K, rho_y=rho, p_y=py, p_z=2 * py,
                                dx=70.0 / max(X, 2))
        out.append((g, synth.tungsten_spectrum(g, lines=k % 2 == 0), synth.random_mask(g, 40 + k)))
    return out


def test_multi_matches_the_oracle_and_the_single_calls(cx):
    caxsi, _, torch = cx
    objs = small_objects()
    plans = [caxsi.Plan(g, phi, mask) for g, phi, mask in objs]
    multi = caxsi.Multi(plans)
    fs = [synth.phantom(g, 10 + k, n_ellipses=3) + 0.05 * synth.uniform_random((g.X, g.J, g.Q), k)
          for k, (g, _, _) in enumerate(objs)]
    ws = [synth.uniform_random((g.M, g.N), 20 + k) + 0.2 for k, (g, _, _) in enumerate(objs)]
    f = multi.pack_f([_t(torch, a) for a in fs])
    w = multi.pack_g([_t(torch, a) for a in ws])
    assert f.numel() == multi.f_len == sum(g.X * g.J * g.Q for g, _, _ in objs)
    assert w.numel() == multi.g_len == sum(g.M * g.N for g, _, _ in objs)
    gm = multi.forward(f)
    fm = multi.adjoint(w)
    D = caxsi.PATH_DIRECT
    for b, ((g, phi, mask), pl) in enumerate(zip(objs, plans)):
        got_g = multi.unpack_g(gm)[b]
        got_f = multi.unpack_f(fm)[b]
        ref_g = oracle.forward(g, phi, mask, _f32(fs[b]))
        ref_f = oracle.adjoint(g, phi, mask, _f32(ws[b]))
        assert rel_l2(got_g.cpu().numpy(), ref_g) <= REL_L2_TOL, b
        assert rel_l2(got_f.cpu().numpy(), ref_f) <= REL_L2_TOL, b
        # the same partial results summed in the same order as the single call
        assert torch.equal(got_g, pl.forward(_t(torch, fs[b]), path=D)), b
        assert torch.equal(got_f, pl.adjoint(_t(torch, ws[b]), path=D)), b
    # repeated launches: the queue hands items out in another order, the sums do not change
    for _ in range(3):
        assert torch.equal(multi.forward(f), gm)
        assert torch.equal(multi.adjoint(w), fm)
    multi.close()
    for pl in plans:
        pl.close()


def test_multi_update_and_reverse_mode_equal_the_single_calls(cx):
    caxsi, _, torch = cx
    objs = small_objects()
    plans = [caxsi.Plan(g, phi, mask) for g, phi, mask in objs]
    multi = caxsi.Multi(plans)
    n = multi.f_len
    rng = np.random.default_rng(9)
    f, b1, b2, c = (torch.tensor(rng.uniform(0.2, 1.5, n), dtype=torch.float32, device="cuda:0")
                    for _ in range(4))
    for beta, delta in ((0.0, 0.1), (0.4, 0.05)):
        out = multi.em_update(f, b1, b2, beta, delta)
        gf, gb2 = multi.em_update_vjp(f, b1, b2, c, beta, delta)
        for b, pl in enumerate(plans):
            sl = slice(int(multi.f_offsets[b]), int(multi.f_offsets[b + 1]))
            ref = pl.em_update(f[sl].contiguous(), b1[sl].contiguous(), b2[sl].contiguous(), beta, delta)
            assert torch.equal(out[sl], ref), (b, beta)
            rf, rb = pl.em_update_vjp(f[sl].contiguous(), b1[sl].contiguous(), b2[sl].contiguous(),
                                      c[sl].contiguous(), beta, delta)
            assert torch.equal(gf[sl], rf) and torch.equal(gb2[sl], rb), (b, beta)
        # against the oracle's update per object
        for b, (g, _, _) in enumerate(objs):
            sl = slice(int(multi.f_offsets[b]), int(multi.f_offsets[b + 1]))
            shp = (g.X, g.J, g.Q)
            ref = oracle.em_update(*(t[sl].double().cpu().numpy().reshape(shp) for t in (f, b1, b2)), beta, delta)
            assert rel_l2(out[sl].cpu().numpy(), ref) <= 1e-6
    with pytest.raises(caxsi.CaxsiError):
        multi.em_update(f, b1, b2, 0.1, 0.1, out=f)       # the output overlaps f
    multi.close()
    for pl in plans:
        pl.close()


def test_multi_errors(cx):
    caxsi, _, torch = cx
    objs = small_objects()[:2]
    plans = [caxsi.Plan(g, phi, mask) for g, phi, mask in objs]
    multi = caxsi.Multi(plans)
    f = torch.zeros(multi.f_len, device="cuda:0")
    with pytest.raises(caxsi.CaxsiError) as e:
        multi.forward(f, path=caxsi.PATH_TABLE_FP32)
    assert e.value.status == 6
    lib, P = multi.lib, __import__("ctypes").c_void_p
    g = torch.zeros(multi.g_len, device="cuda:0")
    assert lib.caxsi_multi_forward(multi.handle, P(f.data_ptr()), multi.f_len - 1, P(g.data_ptr()), multi.g_len,
                                   0, None) == 1
    assert lib.caxsi_multi_adjoint(multi.handle, P(g.data_ptr()), multi.g_len, P(f.data_ptr()), multi.f_len + 1,
                                   0, None) == 1
    assert lib.caxsi_multi_forward(None, P(f.data_ptr()), multi.f_len, P(g.data_ptr()), multi.g_len, 0, None) == 1
    assert lib.caxsi_multi_create(None, 2, None) == 1
    with pytest.raises(caxsi.CaxsiError) as e:       # one plan for two objects: shared scratch
        caxsi.Multi([plans[0], plans[1], plans[0]])
    assert e.value.status == 1
    multi.close()
    for pl in plans:
        pl.close()


def test_unrolled_reconstruction_of_uneven_objects(cx):
    """Unrolled, checkpointed EM over two objects of different (X, J, Q) through the
    packed operator: the gradient equals the per-object gradients of the single-plan
    operator bit for bit, and its directional derivative matches FP64 central finite
    differences of the oracle's iterations."""
    caxsi, autodiff, torch = cx
    shapes = [(16, 16, 16), (12, 16, 24)]
    objs = []
    for k, (X, J, Q) in enumerate(shapes):
        g = synth.make_geometry(X=X, J=J, Q=Q, M=8, N=32, K=8, rho_y=2, p_y=6.08, p_z=12.16, dx=4.375)
        objs.append((g, synth.tungsten_spectrum(g), synth.random_mask(g, 60 + k)))
    plans = [caxsi.Plan(g, phi, mask) for g, phi, mask in objs]
    multi = caxsi.Multi(plans)
    op = autodiff.MultiOperator(multi)
    f_true, ys = [], []
    for k, (g, phi, mask) in enumerate(objs):
        ft = synth.phantom(g, 70 + k, n_ellipses=2)
        mean = oracle.forward(g, phi, mask, ft)
        f_true.append(ft * (300.0 / mean.max()))
        ys.append(synth.poisson_counts(mean * (300.0 / mean.max()), 80 + k))
    beta, delta, n_iter = 0.05, 0.5, 4
    f0s = [np.asarray(np.full(ft.shape, ys[k].sum() / oracle.adjoint(g, phi, mask, np.ones_like(ys[k])).sum())
                      * (1 + 0.2 * synth.uniform_random(ft.shape, 90 + k)), np.float32).astype(np.float64)
           for k, ((g, phi, mask), ft) in enumerate(zip(objs, f_true))]
    y = multi.pack_g([_t(torch, a) for a in ys])
    fT = multi.pack_f([_t(torch, a) for a in f_true]).double()
    f0 = multi.pack_f([_t(torch, a) for a in f0s]).requires_grad_(True)
    out = autodiff.unrolled_em(op, y, f0, n_iter, beta=beta, delta=delta, checkpoint=True)
    torch.sum((out.double() - fT) ** 2).backward()
    grad = f0.grad.double().cpu().numpy()
    # per object through its own plan
    for b, pl in enumerate(plans):
        single = autodiff.Operator(pl, path="direct")
        fb = _t(torch, f0s[b]).requires_grad_(True)
        ob = autodiff.unrolled_em(single, _t(torch, ys[b]), fb, n_iter, beta=beta, delta=delta, checkpoint=True)
        torch.sum((ob.double() - _t(torch, f_true[b]).double()) ** 2).backward()
        sl = slice(int(multi.f_offsets[b]), int(multi.f_offsets[b + 1]))
        assert torch.equal(f0.grad[sl].view_as(fb), fb.grad), b
    # finite differences of the FP64 oracle's iterations, both objects at once

    def L64(x):
        total = 0.0
        for b, (g, phi, mask) in enumerate(objs):
            xb = x[int(multi.f_offsets[b]):int(multi.f_offsets[b + 1])].reshape(g.X, g.J, g.Q)
            A = lambda v, g=g, phi=phi, mask=mask: oracle.forward(g, phi, mask, v)
            At = lambda v, g=g, phi=phi, mask=mask: oracle.adjoint(g, phi, mask, v)
            b1 = oracle.adjoint(g, phi, mask, np.ones_like(ys[b]))
            r = np.zeros_like(ys[b])
            for _ in range(n_iter):
                xb, _ = oracle.em_iteration(A, At, ys[b], r, xb, b1, beta, delta)
            total += float(np.sum((xb - f_true[b]) ** 2))
        return total
    x0 = np.concatenate([a.ravel() for a in f0s])
    d = grad / np.linalg.norm(grad)
    h = 1e-4 * np.linalg.norm(x0)
    fd = (L64(x0 + h * d) - L64(x0 - h * d)) / (2 * h)
    got = float(np.sum(grad * d))
    assert abs(got - fd) <= 1e-3 * abs(fd), (got, fd)
    multi.close()
    for pl in plans:
        pl.close()


# --------------------------------------------------------------------------
# 32 objects of uneven size on the paper-scale detector (256 x 64 pixels,
# 64 energies): the launch configuration the benchmark's batch experiment times
# --------------------------------------------------------------------------

def test_uneven_paper_scale_batch(cx):
    caxsi, _, torch = cx
    base = synth.paper_geometry()
    phi = synth.tungsten_spectrum(base)
    mask = synth.random_mask(base, synth.PAPER_MASK_SEED)
    sizes = synth.uneven_sizes(32, 2024)
    geos = [synth.uneven_object_geometry(X, J, Q) for X, J, Q in sizes]
    assert {g.Q for g in geos} >= {64, 128}
    plans = [caxsi.Plan(g, phi, mask) for g in geos]
    multi = caxsi.Multi(plans)
    D = caxsi.PATH_DIRECT
    fs = [synth.phantom_torch(g, 300 + k, "cuda:0") for k, g in enumerate(geos)]
    gen = torch.Generator(device="cuda:0").manual_seed(5)
    ws = [torch.rand((g.M, g.N), device="cuda:0", generator=gen) + 0.5 for g in geos]
    gm = multi.forward(multi.pack_f(fs))
    fm = multi.adjoint(multi.pack_g(ws))
    for b, pl in enumerate(plans):
        assert torch.equal(multi.unpack_g(gm)[b], pl.forward(fs[b], path=D)), b
        assert torch.equal(multi.unpack_f(fm)[b], pl.adjoint(ws[b], path=D)), b
    # sampled outputs of the smallest, the largest and one other object against the oracle
    rng = np.random.default_rng(11)
    for b in (0, 1, 7):
        g = geos[b]
        pix = np.concatenate([rng.choice(g.M * g.N, 24, replace=False), [0, g.M * g.N - 1]])
        ref = oracle.forward_pixels(g, phi, mask, fs[b].double().cpu().numpy(), pix)
        assert rel_l2(multi.unpack_g(gm)[b].cpu().numpy().ravel()[pix], ref) <= REL_L2_TOL, b
        vox = np.concatenate([rng.choice(g.X * g.J, 12, replace=False), [0, g.X * g.J - 1]])
        refv = oracle.adjoint_voxels(g, phi, mask, ws[b].double().cpu().numpy(), vox)
        got = multi.unpack_f(fm)[b].reshape(g.X * g.J, g.Q).cpu().numpy()[vox]
        assert rel_l2(got, refv) <= REL_L2_TOL, b
    multi.close()
    for pl in plans:
        pl.close()
