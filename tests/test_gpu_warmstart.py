"""The learned warm start's kernels (include/caxsi_nn.h) and network.

References: plain PyTorch CPU operators in float64 (convolution, pooling,
upsampling, autograd) with the same bf16 rounding of the convolution inputs as
the tensor-core GEMMs; tolerances cover bf16 rounding of the backward operands
(relative L2 <= 3e-2 for gradients) and FP32 accumulation elsewhere.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    import torch
    from paper_1603_06400_gb300 import build, caxsi, warmstart
    build.build()
    return torch, caxsi, warmstart


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _rb(torch, t):
    return t.to(torch.bfloat16).to(torch.float64)


def _conv_weight(torch, layer):
    W = layer.W.w.detach().cpu().double()
    return W.view(layer.cout, layer.k, layer.k, layer.cin).permute(0, 3, 1, 2).contiguous()


def test_conv3x3_forward_and_backward(ws):
    torch, caxsi, warmstart = ws
    import torch.nn.functional as F
    gen = torch.Generator().manual_seed(3)
    n, H, W, cin, cout = 2, 6, 10, 16, 24
    K = warmstart._Ops()
    layer = warmstart.Conv(cin, cout, 3, True, gen)
    layer.b.w.copy_(torch.linspace(-0.2, 0.3, cout))
    x = torch.randn(n * H * W, cin, generator=gen).cuda()
    y = layer.forward(K, x, n, H, W)
    dy = torch.randn(n * H * W, cout, generator=gen).cuda()
    dx = layer.backward(K, dy.clone())
    torch.cuda.synchronize()
    # reference
    xr = x.cpu().double().view(n, H, W, cin).permute(0, 3, 1, 2).requires_grad_(True)
    Wr = _conv_weight(torch, layer).requires_grad_(True)
    br = layer.b.w.cpu().double().requires_grad_(True)
    yr = F.relu(F.conv2d(_rb(torch, xr), _rb(torch, Wr), br, padding=1))
    yr.backward(dy.cpu().double().view(n, H, W, cout).permute(0, 3, 1, 2))
    assert rel_l2(y.cpu(), yr.permute(0, 2, 3, 1).reshape(-1, cout).detach()) <= 1e-5
    assert rel_l2(layer.b.g.cpu(), br.grad) <= 1e-5
    gW = Wr.grad.permute(0, 2, 3, 1).reshape(cout, 9 * cin)
    assert rel_l2(layer.W.g.cpu(), gW) <= 3e-2
    assert rel_l2(dx.cpu(), xr.grad.permute(0, 2, 3, 1).reshape(-1, cin)) <= 3e-2


def test_pool_upsample_copy_mse_adam(ws):
    torch, caxsi, warmstart = ws
    import torch.nn.functional as F
    K = warmstart._Ops()
    P = warmstart._p
    gen = torch.Generator().manual_seed(4)
    n, H, W, C = 2, 4, 6, 8
    x = torch.randn(n, H, W, C, generator=gen).cuda()
    y = torch.empty(n, H // 2, W // 2, C, device="cuda")
    K("pool2", P(x), n, H, W, C, P(y))
    ref = F.avg_pool2d(x.cpu().permute(0, 3, 1, 2), 2).permute(0, 2, 3, 1)
    assert torch.allclose(y.cpu(), ref, atol=1e-6)
    d = torch.randn_like(y)
    dx = torch.empty_like(x)
    K("pool2_bwd", P(d), n, H, W, C, P(dx))
    assert torch.allclose(dx.cpu(), d.cpu().repeat_interleave(2, 1).repeat_interleave(2, 2) / 4, atol=1e-7)
    u = torch.empty(n, 2 * H, 2 * W, C, device="cuda")
    K("up2", P(x), n, H, W, C, P(u))
    assert torch.equal(u.cpu(), x.cpu().repeat_interleave(2, 1).repeat_interleave(2, 2))
    du = torch.randn_like(u)
    dxu = torch.empty_like(x)
    K("up2_bwd", P(du), n, H, W, C, P(dxu))
    ref = du.cpu().view(n, H, 2, W, 2, C).sum((2, 4))
    assert torch.allclose(dxu.cpu(), ref, atol=1e-5)
    cat = torch.zeros(n * H * W, 3 * C, device="cuda")
    K("copy_channels", P(x), n * H * W, C, 0, C, P(cat), C, 3 * C)
    assert torch.equal(cat[:, C:2 * C].cpu(), x.view(-1, C).cpu()) and float(cat[:, :C].abs().sum()) == 0.0
    t = torch.randn_like(x)
    grad = torch.empty_like(x)
    K("mse", P(x), P(t), x.numel(), P(grad), P(K.loss))
    assert float(K.loss[0]) == pytest.approx(float(((x - t).double() ** 2).mean()), rel=1e-12)
    assert torch.allclose(grad, 2 * (x - t) / x.numel(), atol=1e-9)
    w = torch.randn(100, generator=gen).cuda()
    g = torch.randn(100, generator=gen).cuda()
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    w0 = w.clone()
    opt = torch.optim.Adam([w0.cpu().requires_grad_(True)], lr=1e-2)
    p = opt.param_groups[0]["params"][0]
    for step in range(1, 4):
        K("adam", P(w), P(g), P(m), P(v), 100, 1e-2, 0.9, 0.999, 1e-8, step)
        p.grad = g.cpu().clone()
        opt.step()
    assert torch.allclose(w.cpu(), p.detach(), atol=1e-6)


def _ref_unet(torch, net, x, n, H, W):
    """The same network in float64 PyTorch CPU ops (bf16-rounded conv inputs)."""
    import torch.nn.functional as F
    Ws = {}

    def conv(layer, h, relu):
        Wc = _conv_weight(torch, layer).requires_grad_(True)
        b = layer.b.w.detach().cpu().double().requires_grad_(True)
        Ws[id(layer)] = (Wc, b)
        out = F.conv2d(_rb(torch, h), _rb(torch, Wc), b, padding=layer.k // 2)
        return F.relu(out) if relu else out
    C = net.channels
    h0 = x.cpu().double().view(n, H, W, C).permute(0, 3, 1, 2)
    skips, h = [], h0
    for lvl, (ca, cb) in enumerate(net.enc):
        h = conv(cb, conv(ca, h, True), True)
        if lvl < 3:
            skips.append(h)
            h = F.avg_pool2d(h, 2)
    for lvl in (2, 1, 0):
        cu, ca, cb = net.dec[lvl]
        t = conv(cu, F.interpolate(h, scale_factor=2, mode="nearest"), True)
        h = conv(cb, conv(ca, torch.cat([t, skips[lvl]], 1), True), True)
    out = conv(net.head, h, False) + h0
    return out, Ws


def test_unet_forward_and_gradients(ws):
    torch, caxsi, warmstart = ws
    n, H, W, C = 1, 16, 32, 16
    net = warmstart.UNet(channels=C, base=8, seed=1)
    gen = torch.Generator().manual_seed(5)
    x = torch.rand(n * H * W, C, generator=gen).cuda()
    tgt = torch.rand(n * H * W, C, generator=gen).cuda()
    out = net.forward(x, n, H, W)
    loss, grad = net.mse(out, tgt)
    net.backward(grad)
    torch.cuda.synchronize()
    ref, Ws = _ref_unet(torch, net, x, n, H, W)
    refo = ref.permute(0, 2, 3, 1).reshape(-1, C)
    assert rel_l2(out.cpu(), refo.detach()) <= 2e-3
    lr = ((refo - tgt.cpu().double()) ** 2).mean()
    assert float(loss) == pytest.approx(float(lr.detach()), rel=1e-2)
    lr.backward()
    for layer in net.layers():
        Wc, b = Ws[id(layer)]
        gW = Wc.grad.permute(0, 2, 3, 1).reshape(layer.cout, -1)
        assert rel_l2(layer.W.g.cpu(), gW) <= 5e-2, (layer.cin, layer.cout)
        assert rel_l2(layer.b.g.cpu(), b.grad) <= 5e-2


def test_warm_start_training_lowers_the_loss(ws, tiny):
    torch, caxsi, warmstart = ws
    g, phi, mask = tiny
    plan = caxsi.Plan(g, phi, mask)
    maker = warmstart.PairMaker(plan, g)
    net = warmstart.UNet(channels=g.Q, base=8, seed=2)
    f1, f_ref, *_ = maker.make(123)
    s = float(f1.mean())
    x = (f1 / s).view(-1, g.Q).contiguous()
    tgt = (f_ref / s).view(-1, g.Q).contiguous()
    first = None
    for k in range(40):
        out = net.forward(x, 1, g.X, g.J)
        loss, grad = net.mse(out, tgt)
        first = float(loss) if first is None else first
        net.backward(grad)
        net.step(2e-3)
    last = float(net.mse(net.forward(x, 1, g.X, g.J), tgt)[0])
    assert last < 0.97 * first, (first, last)
    f0 = net.predict(f1, s, 1e-6 * s)
    assert bool(torch.isfinite(f0).all()) and float(f0.min()) >= 1e-6 * s * (1 - 1e-6)
    assert int(net.K.err[0]) == 0
    plan.close()


def test_step_scalings_train_and_unit_scalings_are_plain_iterations(ws, tiny):
    torch, caxsi, warmstart = ws
    g, phi, mask = tiny
    plan = caxsi.Plan(g, phi, mask)
    maker = warmstart.PairMaker(plan, g)
    net = warmstart.UNet(channels=g.Q, base=8, seed=3)
    relax = warmstart.train_step_scalings(net, maker, T=3, samples=3)
    assert relax.shape == (3,) and bool(torch.isfinite(relax).all())
    # unit scalings are the plain EM-type iterations of caxsi_recon_step
    f1, f_ref, y, beta, delta, _ = maker.make(7)
    f_a = warmstart.relaxed_iterations(maker, y, f1.clone(), torch.ones(3, device="cuda"), beta, delta, 0.0)
    f_b = f1.clone()
    for _ in range(3):
        plan.recon_step(y, f_b, beta=beta, delta=delta, path=caxsi.PATHS["table_fp32"])
    assert torch.allclose(f_a, f_b, rtol=1e-5, atol=1e-6 * float(f_b.abs().max()))
    plan.close()


def test_trained_warm_start_beats_the_flat_start_on_held_out_objects(ws, tiny):
    """Train briefly (200 steps of 4 objects, seeds 100000+), then on 6 held-out
    objects (seeds 900000+, never trained on): after the same number T = 20 of
    EM-type iterations, the warm-started reconstruction has a lower NMSE than the
    flat-started one for every object, by 10 % on average, and reaches the flat
    start's final NMSE in fewer iterations.  The held-out loss falls during training."""
    torch, caxsi, warmstart = ws
    g, phi, mask = tiny
    plan = caxsi.Plan(g, phi, mask)
    maker = warmstart.PairMaker(plan, g)
    net = warmstart.UNet(channels=g.Q, base=16, seed=0)
    losses = warmstart.train(net, maker, 200, lr=1e-3, batch=4, log=50, heldout_seeds=range(150000, 150004))
    assert losses[-1][2] < losses[0][2], losses
    P = caxsi.PATHS["table_fp32"]
    T = 20
    ratios = []
    for k in range(6):
        f1, f_ref, y, beta, delta, _ = maker.make(900000 + k)
        nref = float((f_ref.double() ** 2).sum())
        nmse = lambda f: float(((f.double() - f_ref.double()) ** 2).sum()) / nref
        flat = f1.clone()              # the first iterate from the flat start is iteration 1
        for _ in range(T - 1):
            plan.recon_step(y, flat, beta=beta, delta=delta, path=P)
        target = nmse(flat)
        s = float(f1.mean())
        warm = net.predict(f1, s, 1e-3 * s)
        hist = [nmse(warm)]
        for _ in range(T - 1):
            plan.recon_step(y, warm, beta=beta, delta=delta, path=P)
            hist.append(nmse(warm))
        assert hist[-1] < target, (k, hist[-1], target)
        reach = next(i for i, v in enumerate(hist) if v <= target)
        assert reach < T - 1, (k, reach)
        ratios.append(hist[-1] / target)
    assert float(np.mean(ratios)) < 0.9, ratios
    plan.close()


def test_device_poisson_draws(ws):
    """caxsi_nn_poisson: integer draws whose mean and variance match the Poisson
    law over both samplers (inversion below 10, transformed rejection above),
    a chi-square fit of the frequencies, and reproducibility by seed."""
    import ctypes
    torch, caxsi, warmstart = ws
    lib = caxsi.load()
    P = warmstart._p

    def draw(lam, n, seed, scale=1.0):
        mean = torch.full((n,), lam, device="cuda")
        y = torch.empty_like(mean)
        assert lib.caxsi_nn_poisson(P(mean), ctypes.c_float(scale), n, ctypes.c_uint64(seed), P(y), None) == 0
        return y
    n = 200000
    for lam in (0.0, 0.3, 3.0, 9.5, 10.0, 57.0, 1000.0, 1e4):
        y = draw(lam, n, 7).double().cpu().numpy()
        assert np.all(y == np.round(y)) and y.min() >= 0
        if lam == 0.0:
            assert y.max() == 0
            continue
        assert abs(y.mean() - lam) <= 5 * np.sqrt(lam / n), lam
        assert abs(y.var() / lam - 1) <= 5 * np.sqrt(2.0 / n) + 2e-3, lam
    from scipy import stats
    for lam in (3.0, 57.0):
        y = draw(lam, n, 11).cpu().numpy().astype(np.int64)
        lo, hi = int(stats.poisson.ppf(1e-4, lam)), int(stats.poisson.ppf(1 - 1e-4, lam))
        obs = np.array([np.sum(y <= lo)] + [np.sum(y == k) for k in range(lo + 1, hi)] + [np.sum(y >= hi)])
        pk = np.array([stats.poisson.cdf(lo, lam)] + [stats.poisson.pmf(k, lam) for k in range(lo + 1, hi)] +
                      [stats.poisson.sf(hi - 1, lam)])
        chi2 = float(np.sum((obs - n * pk) ** 2 / (n * pk)))
        assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-4, (lam, chi2)
    a, b, c = draw(5.0, 4096, 1), draw(5.0, 4096, 1), draw(5.0, 4096, 2)
    assert torch.equal(a, b) and not torch.equal(a, c)
    # the scale multiplies the mean
    assert torch.equal(draw(2.5, 4096, 3, scale=2.0), draw(5.0, 4096, 3))
