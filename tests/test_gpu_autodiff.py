"""Batched operators and automatic differentiation through the C ABI.

- Batches of objects of uneven size (voxel ranges of one geometry): each
  object's result is bit-identical to the single-object call, and matches the
  FP64 oracle.
- A / A^T under autograd, the EM update's reverse-mode kernel and the unrolled
  (checkpointed) reconstruction: directional derivatives against FP64 central
  finite differences of the same functions evaluated by the oracle, on a
  16 x 16 x 16 object.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def cx():
    import torch
    from paper_1603_06400_gb300 import autodiff, build, caxsi
    build.build()
    return caxsi, autodiff, torch


def _t(torch, a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda:0")


def geom16():
    """A 16 x 16 x 16 object (X, J, Q) with an 8 x 32 detector and 8 energies,
    spanning the paper's 70 x 194.6 mm field and 194.6 x 97.3 mm detector."""
    return synth.make_geometry(X=16, J=16, Q=16, M=8, N=32, K=8, rho_y=2, p_y=6.08, p_z=12.16,
                               dx=4.375)


# ---------------------------------------------------------------------------
# batches of objects of uneven size
# ---------------------------------------------------------------------------

def _uneven_ranges(R, nb, seed):
    rng = np.random.default_rng(seed)
    out = []
    for b in range(nb):
        if b == 0:
            out.append((0, R))           # the whole field
        elif b == 1:
            out.append((R // 3, R // 3))   # an empty object
        else:
            a, c = sorted(rng.integers(0, R + 1, size=2))
            out.append((int(a), int(c)))
    return np.array(out, np.int32)


@pytest.mark.parametrize("nb", [1, 5, 32])
def test_batch_is_exactly_the_single_calls(cx, tiny, nb):
    caxsi, _, torch = cx
    g, phi, mask = tiny
    R = g.X * g.J
    plan = caxsi.Plan(g, phi, mask)
    plan.set_symmetry(False)   # batches stream one record per open pair, as these single calls then do
    ranges = _uneven_ranges(R, nb, 10 + nb)
    f = torch.rand((nb, g.X, g.J, g.Q), device="cuda:0")
    w = torch.rand((nb, g.M, g.N), device="cuda:0") + 0.1
    gb = plan.forward_batch(f, ranges=ranges)
    fb = plan.adjoint_batch(w, ranges=ranges)
    P = caxsi.PATHS["table_fp32"]
    for b, (v0, v1) in enumerate(ranges):
        fo = torch.zeros_like(f[b]).view(R, g.Q)
        fo[v0:v1] = f[b].view(R, g.Q)[v0:v1]
        assert torch.equal(gb[b], plan.forward(fo.view(g.X, g.J, g.Q).contiguous(), path=P)), b
        full = plan.adjoint(w[b].contiguous(), path=P).view(R, g.Q)
        got = fb[b].view(R, g.Q)
        assert torch.equal(got[v0:v1], full[v0:v1]), b
        assert torch.count_nonzero(got[:v0]) == 0 and torch.count_nonzero(got[v1:]) == 0, b
    assert plan.info()["device_error"] == 0
    plan.close()


def test_batch_matches_the_oracle(cx):
    caxsi, _, torch = cx
    g = synth.make_geometry(X=5, J=7, Q=37, M=9, N=45, K=13, rho_y=3, p_y=2.5, p_z=4.0, dx=6.0)
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 77)
    R = g.X * g.J
    plan = caxsi.Plan(g, phi, mask)
    ranges = np.array([[3, 29], [0, R]], np.int32)
    f = synth.uniform_random((2, g.X, g.J, g.Q), 8)
    w = synth.uniform_random((2, g.M, g.N), 9) + 0.2
    gb = plan.forward_batch(_t(torch, f), ranges=ranges).cpu().numpy()
    fb = plan.adjoint_batch(_t(torch, w), ranges=ranges).cpu().numpy()
    for b, (v0, v1) in enumerate(ranges):
        fm = np.zeros((R, g.Q))
        fm[v0:v1] = np.asarray(f[b], np.float32).reshape(R, g.Q)[v0:v1]
        ref_g = oracle.forward(g, phi, mask, fm.reshape(g.X, g.J, g.Q))
        assert rel_l2(gb[b], ref_g) <= 1e-5
        ref_f = oracle.adjoint(g, phi, mask, np.asarray(w[b], np.float32).astype(np.float64)).reshape(R, g.Q)
        assert rel_l2(fb[b].reshape(R, g.Q)[v0:v1], ref_f[v0:v1]) <= 1e-5
    plan.close()


def test_batch_rejects_bad_layouts(cx, tiny):
    caxsi, _, torch = cx
    g, phi, mask = tiny
    plan = caxsi.Plan(g, phi, mask)
    f = torch.rand((2, g.X, g.J, g.Q), device="cuda:0")
    for bad in ([[0, 5], [6, 5]], [[-1, 3], [0, 1]], [[0, g.X * g.J + 1], [0, 1]]):
        with pytest.raises(caxsi.CaxsiError) as e:
            plan.forward_batch(f, ranges=bad)
        assert e.value.status == 1
    with pytest.raises(caxsi.CaxsiError) as e:   # the batch is an FP32 table-path call
        plan.forward_batch(f, path=caxsi.PATHS["table_bf16"])
    assert e.value.status == 6
    plan.close()


# ---------------------------------------------------------------------------
# automatic differentiation against FP64 finite differences (oracle)
# ---------------------------------------------------------------------------

def _problem16(seed=0):
    g = geom16()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 300 + seed)
    f_true = synth.phantom(g, seed, n_ellipses=3)
    mean = oracle.forward(g, phi, mask, f_true)
    y = synth.poisson_counts(mean * (300.0 / mean.max()), 40 + seed)
    return g, phi, mask, f_true * (300.0 / mean.max()), y


def _fd(fun, x, d, h):
    return (fun(x + h * d) - fun(x - h * d)) / (2.0 * h)


def test_operator_gradient_of_the_likelihood(cx):
    caxsi, autodiff, torch = cx
    g, phi, mask, f_true, y = _problem16(0)
    plan = caxsi.Plan(g, phi, mask)
    op = autodiff.Operator(plan)
    r = 0.5
    f0 = np.asarray(f_true + 0.3 * synth.uniform_random(f_true.shape, 1), np.float32).astype(np.float64)
    ft = _t(torch, f0).requires_grad_(True)
    z = op(ft) + r
    yt = _t(torch, y)
    L = torch.sum(z.double() - yt.double() * torch.log(z.double()))
    L.backward()
    grad = ft.grad.double().cpu().numpy()

    def L64(f):
        zz = oracle.forward(g, phi, mask, f) + r
        return float(np.sum(zz - y * np.log(zz)))
    # along the gradient itself (no cancellation in the dot product)
    d = grad / np.linalg.norm(grad)
    assert rel(float(np.sum(grad * d)), _fd(L64, f0, d, 1e-3)) <= 1e-5
    # random directions: dL = sum_i (1 - y_i / z_i) (A d)_i cancels heavily, and
    # z carries FP32 rounding, so the error is bounded on the scale of the terms
    zz = oracle.forward(g, phi, mask, f0) + r
    for k in range(3):
        d = synth.normal_random(f0.shape, 50 + k)
        scale = float(np.sum(np.abs(oracle.forward(g, phi, mask, d)) * (1.0 + y / zz)))
        err = abs(float(np.sum(grad * d)) - _fd(L64, f0, d, 1e-4))
        assert err <= 1e-5 * scale, (k, err, scale)
    plan.close()


def test_update_reverse_mode(cx):
    caxsi, _, torch = cx
    g = geom16()
    plan = caxsi.Plan(g, synth.tungsten_spectrum(g), synth.random_mask(g, 5))
    shape = (g.X, g.J, g.Q)
    f = np.asarray(0.5 + synth.uniform_random(shape, 1), np.float32).astype(np.float64)
    b1 = np.asarray(0.5 + synth.uniform_random(shape, 2), np.float32).astype(np.float64)
    b2 = np.asarray(0.5 + synth.uniform_random(shape, 3), np.float32).astype(np.float64)
    c = synth.normal_random(shape, 4)
    for beta, delta in ((0.0, 0.1), (0.3, 0.05), (2.0, 0.4)):
        got = plan.em_update(_t(torch, f), _t(torch, b1), _t(torch, b2), beta, delta).cpu().numpy()
        assert rel_l2(got, oracle.em_update(f, b1, b2, beta, delta)) <= 1e-6
        gf, gb2 = plan.em_update_vjp(_t(torch, f), _t(torch, b1), _t(torch, b2), _t(torch, c), beta, delta)
        gf, gb2 = gf.double().cpu().numpy(), gb2.double().cpu().numpy()
        Lf = lambda x: float(np.sum(c * oracle.em_update(x, b1, b2, beta, delta)))
        Lb = lambda x: float(np.sum(c * oracle.em_update(f, b1, x, beta, delta)))
        for k in range(3):
            d = synth.normal_random(shape, 20 + k)
            assert rel(float(np.sum(gf * d)), _fd(Lf, f, d, 1e-6)) <= 1e-4, (beta, k)
            assert rel(float(np.sum(gb2 * d)), _fd(Lb, b2, d, 1e-6)) <= 1e-4, (beta, k)
    plan.close()


def test_unrolled_reconstruction_gradient(cx):
    caxsi, autodiff, torch = cx
    g, phi, mask, f_true, y = _problem16(1)
    plan = caxsi.Plan(g, phi, mask)
    op = autodiff.Operator(plan)
    r = np.full_like(y, 0.2)
    beta, delta, n_iter = 0.05, 0.5, 10
    b1 = oracle.adjoint(g, phi, mask, np.ones_like(y))
    f0 = np.asarray(np.full(f_true.shape, y.sum() / b1.sum()) * (1 + 0.2 * synth.uniform_random(f_true.shape, 6)),
                    np.float32).astype(np.float64)
    yt, rt = _t(torch, y), _t(torch, r)
    ft = _t(torch, f0).requires_grad_(True)
    fT = _t(torch, f_true).double()
    out = autodiff.unrolled_em(op, yt, ft, n_iter, r=rt, beta=beta, delta=delta, checkpoint=True)
    L = torch.sum((out.double() - fT) ** 2)
    L.backward()
    grad = ft.grad.double().cpu().numpy()
    # the same gradient without checkpointing (deterministic kernels: identical)
    ft2 = _t(torch, f0).requires_grad_(True)
    out2 = autodiff.unrolled_em(op, yt, ft2, n_iter, r=rt, beta=beta, delta=delta, checkpoint=False)
    torch.sum((out2.double() - fT) ** 2).backward()
    assert torch.equal(ft.grad, ft2.grad)

    A = lambda x: oracle.forward(g, phi, mask, x)
    At = lambda x: oracle.adjoint(g, phi, mask, x)

    def L64(x):
        for _ in range(n_iter):
            x, _ = oracle.em_iteration(A, At, y, r, x, b1, beta, delta)
        return float(np.sum((x - f_true) ** 2))
    # along the gradient (relative), and along random directions on the scale
    # of the terms of the dot product (10 FP32 iterations against FP64)
    d = grad / np.linalg.norm(grad)
    got, fd = float(np.sum(grad * d)), _fd(L64, f0, d, 1e-4 * np.linalg.norm(f0))
    assert rel(got, fd) <= 1e-3, (got, fd)
    for k in range(2):
        d = synth.normal_random(f0.shape, 70 + k) * f0
        got, fd = float(np.sum(grad * d)), _fd(L64, f0, d, 1e-5)
        assert abs(got - fd) <= 1e-3 * float(np.sum(np.abs(grad * d))), (k, got, fd)
    plan.close()


def test_checkpointing_lowers_peak_memory(cx, tiny):
    caxsi, autodiff, torch = cx
    g, phi, mask = tiny
    plan = caxsi.Plan(g, phi, mask)
    op = autodiff.Operator(plan)
    y = torch.rand((g.M, g.N), device="cuda:0") * 50
    peaks = {}
    for ck in (False, True):
        f0 = torch.full((g.X, g.J, g.Q), 0.5, device="cuda:0", requires_grad=True)
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        out = autodiff.unrolled_em(op, y, f0, 10, beta=0.01, delta=0.1, checkpoint=ck)
        out.sum().backward()
        torch.cuda.synchronize()
        peaks[ck] = torch.cuda.max_memory_allocated() - base
    # without checkpointing each iteration keeps its input and A^T(ratio) (two
    # object-sized tensors); with it, only its input
    assert peaks[True] < 0.75 * peaks[False], peaks
    plan.close()


def test_ratio_and_its_reverse_mode(cx, tiny):
    """caxsi_ratio / caxsi_ratio_vjp against the definitions in FP64, with the edge
    rules: z <= 0 gives ratio 0 and derivative 0; a positive count there sets the
    error word that the next likelihood call reports."""
    caxsi, _, torch = cx
    g, phi, mask = tiny
    plan = caxsi.Plan(g, phi, mask)
    n = 3 * g.M * g.N + 5      # any length: images back to back and a ragged tail
    rng = np.random.default_rng(3)
    gg = rng.uniform(0.1, 4.0, n).astype(np.float32)
    y = rng.poisson(3.0, n).astype(np.float32)
    r = rng.uniform(0.0, 0.5, n).astype(np.float32)
    gg[:7] = [0.0, -1.0, 0.0, -0.5, 2.0, 0.0, -0.25]
    r[:7] = [0.0, 0.5, 0.0, 0.0, 0.0, 0.0, 0.0]
    y[:7] = [0.0, 0.0, 0.0, 0.0, 5.0, 0.0, 0.0]
    gr = rng.normal(size=n).astype(np.float32)
    for rr in (None, r):
        z = gg.astype(np.float64) + (0.0 if rr is None else rr.astype(np.float64))
        want = np.where(z > 0, y / np.where(z > 0, z, 1.0), 0.0)
        dwant = np.where(z > 0, -gr * y / np.where(z > 0, z, 1.0) ** 2, 0.0)
        rt = None if rr is None else _t(torch, rr)
        got = plan.ratio(_t(torch, gg), _t(torch, y), rt).double().cpu().numpy()
        dgot = plan.ratio_vjp(_t(torch, gg), _t(torch, y), _t(torch, gr), rt).double().cpu().numpy()
        np.testing.assert_allclose(got, want, rtol=2e-7, atol=0)
        np.testing.assert_allclose(dgot, dwant, rtol=1e-6, atol=0)
        assert np.all(got[z <= 0] == 0) and np.all(dgot[z <= 0] == 0)
    # no positive count met z <= 0 so far: a likelihood call succeeds
    zero_counts = torch.zeros((g.M, g.N), device="cuda:0")    # no count can meet z <= 0
    f = torch.full((g.X, g.J, g.Q), 0.1, device="cuda:0")
    plan.recon_step(zero_counts, f.clone(), want_nll=True)
    bad_y = y.copy()
    bad_y[1] = 2.0          # z = -1 + 0.5 < 0 with a positive count
    plan.ratio(_t(torch, gg), _t(torch, bad_y), _t(torch, r))
    with pytest.raises(caxsi.CaxsiError) as e:
        plan.recon_step(zero_counts, f.clone(), want_nll=True)
    assert e.value.status == 4
    plan.recon_step(zero_counts, f.clone(), want_nll=True)     # the word is cleared once reported
    plan.close()


def test_update_rejects_overlapping_outputs(cx):
    caxsi, _, torch = cx
    g = geom16()
    plan = caxsi.Plan(g, synth.tungsten_spectrum(g), synth.random_mask(g, 5))
    shape = (g.X, g.J, g.Q)
    f, b1, b2, c = (torch.rand(shape, device="cuda:0") + 0.5 for _ in range(4))
    with pytest.raises(caxsi.CaxsiError) as e:
        plan.em_update(f, b1, b2, 0.1, 0.1, out=f)          # in place
    assert e.value.status == 1
    # a buffer that overlaps f by one element
    big = torch.rand(2 * f.numel(), device="cuda:0") + 0.5
    fa, fb = big[: f.numel()].view(shape), big[f.numel() - 1: 2 * f.numel() - 1].view(shape)
    with pytest.raises(caxsi.CaxsiError):
        plan.em_update(fa, b1, b2, 0.1, 0.1, out=fb)
    lib, P = plan.lib, ctypes.c_void_p
    n = f.numel()
    # reverse mode: grad_f on top of an input or of grad_b2
    for gf_t, gb_t in ((f, c.clone()), (c.clone(), b2), (b1.clone(), None)):
        gb_t = gf_t if gb_t is None else gb_t
        st = lib.caxsi_em_update_vjp(plan.handle, P(f.data_ptr()), P(b1.data_ptr()), P(b2.data_ptr()), 0.1, 0.1,
                                     P(c.data_ptr()), P(gf_t.data_ptr()), P(gb_t.data_ptr()), n, None)
        assert st == 1
    # disjoint buffers are accepted and give the same result as before
    out = plan.em_update(f, b1, b2, 0.1, 0.1)
    assert torch.isfinite(out).all()
    plan.close()
