"""Learned warm start for the EM-type reconstruction (an extension: the paper
has no learned component).

A 2-D U-Net over the object's (i, j) plane, with the Q = 128 q bins as
channels, maps the first EM-type iterate (Algorithm 4 from a flat start) to a
starting image f^0; the EM-type iterations then continue from f^0.  Four
levels with base width 32 (32, 64, 128, 256 channels), two 3x3 convolutions
with ReLU per level, 2x2 average pooling, nearest upsampling followed by a 3x3
convolution, skip connections by channel concatenation, and a 1x1 output
convolution added to the input.  Every layer runs in the library's kernels
(include/caxsi_nn.h): convolutions as im2col plus bf16 tensor-core GEMMs with
FP32 accumulation, backward passes by the same GEMMs, Adam updates.  Training
pairs come from the forward model with Poisson noise on phantoms of the
synthetic-input recipe, generated on the fly.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import caxsi

BF16 = torch.bfloat16


def _p(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else None)


class _Ops:
    """Status-checked calls of caxsi_nn_* on the current torch stream."""

    def __init__(self):
        self.lib = caxsi.load()
        self.err = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.loss = torch.zeros(1 + 512, dtype=torch.float64, device="cuda")

    def __call__(self, name, *args):
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        caxsi._check(getattr(self.lib, "caxsi_nn_" + name)(*args, s), "caxsi_nn_" + name)

    def gemm(self, M, N, K, A, B, C):
        """C[M][N] = A[M][K] B[N][K]^T (bf16 operands, FP32 out)."""
        self("gemm_bf16", M, N, K, _p(A), _p(B), _p(C), _p(self.err))

    def bf16(self, x):
        y = torch.empty(x.shape, dtype=BF16, device=x.device)
        self("to_bf16", _p(x), _p(y), x.numel())
        return y

    def transpose(self, x, rows, cols):
        y = torch.empty((cols, rows), dtype=BF16, device=x.device)
        self("transpose_bf16", _p(x), int(x.dtype == torch.float32), rows, cols, _p(y))
        return y


class _Param:
    def __init__(self, w):
        self.w = w
        self.g = torch.zeros_like(w)
        self.m = torch.zeros_like(w)
        self.v = torch.zeros_like(w)


class Conv:
    """k x k 'same' convolution (k = 3 or 1) on NHWC FP32 activations, optional ReLU."""

    def __init__(self, cin, cout, k, relu, gen, scale=None):
        fan = k * k * cin
        std = math.sqrt(2.0 / fan) if scale is None else scale
        self.W = _Param((torch.randn(cout, fan, generator=gen, dtype=torch.float64) * std).float().cuda())
        self.b = _Param(torch.zeros(cout, device="cuda"))
        self.cin, self.cout, self.k, self.relu = cin, cout, k, relu

    def params(self):
        return [self.W, self.b]

    def forward(self, K, x, n, H, W):
        P = n * H * W
        self.shape = (n, H, W)
        if self.k == 3:
            col = torch.empty((P, 9 * self.cin), dtype=BF16, device="cuda")
            K("im2col3x3", _p(x), n, H, W, self.cin, _p(col))
        else:
            col = K.bf16(x)
        y = torch.empty((P, self.cout), device="cuda")
        K.gemm(P, self.cout, self.k * self.k * self.cin, col, K.bf16(self.W.w), y)
        K("bias_act", _p(y), _p(self.b.w), P, self.cout, int(self.relu))
        self.col, self.y = col, y
        return y

    def backward(self, K, dy, need_dx=True):
        n, H, W = self.shape
        P, kk = n * H * W, self.k * self.k * self.cin
        if self.relu:
            K("relu_bwd", _p(dy), _p(self.y), dy.numel())
        K("bias_grad", _p(dy), P, self.cout, _p(self.b.g))
        K.gemm(self.cout, kk, P, K.transpose(dy, P, self.cout), K.transpose(self.col, P, kk), self.W.g)
        if not need_dx:
            return None
        dcol = torch.empty((P, kk), device="cuda")
        K.gemm(P, kk, self.cout, K.bf16(dy), K.transpose(self.W.w, self.cout, kk), dcol)
        if self.k == 1:
            return dcol
        dx = torch.empty((P, self.cin), device="cuda")
        K("col2im3x3", _p(dcol), n, H, W, self.cin, _p(dx))
        return dx


class UNet:
    """The warm-start network; activations [n*H*W][C] for an object batch [n][H][W][C]."""

    def __init__(self, channels: int = 128, base: int = 32, seed: int = 0):
        gen = torch.Generator().manual_seed(seed)
        c1, c2, c3, c4 = base, 2 * base, 4 * base, 8 * base
        C = lambda ci, co, relu=True: Conv(ci, co, 3, relu, gen)
        self.enc = [(C(channels, c1), C(c1, c1)), (C(c1, c2), C(c2, c2)), (C(c2, c3), C(c3, c3)),
                    (C(c3, c4), C(c4, c4))]
        # decoder level l: upsampling conv (c_{l+1} -> c_l), then two convs on [up | skip]
        self.dec = [(C(c2, c1), C(2 * c1, c1), C(c1, c1)), (C(c3, c2), C(2 * c2, c2), C(c2, c2)),
                    (C(c4, c3), C(2 * c3, c3), C(c3, c3))]
        self.head = Conv(c1, channels, 1, False, gen, scale=1e-3)
        self.widths = (c1, c2, c3, c4)
        self.channels = channels
        self.K = _Ops()
        self.t = 0

    def layers(self):
        out = [c for pair in self.enc for c in pair] + [c for tri in self.dec for c in tri] + [self.head]
        return out

    def forward(self, x, n, H, W):
        """x: [n*H*W][channels] -> x + head(...), same shape."""
        K, w = self.K, self.widths
        self.sizes = [(H >> l, W >> l) for l in range(4)]
        self.n = n
        skips, h = [], x
        for lvl, (ca, cb) in enumerate(self.enc):
            hh, ww = self.sizes[lvl]
            h = cb.forward(K, ca.forward(K, h, n, hh, ww), n, hh, ww)
            if lvl < 3:
                skips.append(h)
                pooled = torch.empty((n * (hh // 2) * (ww // 2), w[lvl]), device="cuda")
                K("pool2", _p(h), n, hh, ww, w[lvl], _p(pooled))
                h = pooled
        for lvl in (2, 1, 0):
            cu, ca, cb = self.dec[lvl]
            hh, ww = self.sizes[lvl]
            up = torch.empty((n * hh * ww, w[lvl + 1]), device="cuda")
            K("up2", _p(h), n, hh // 2, ww // 2, w[lvl + 1], _p(up))
            t = cu.forward(K, up, n, hh, ww)
            cat = torch.empty((n * hh * ww, 2 * w[lvl]), device="cuda")
            P = n * hh * ww
            K("copy_channels", _p(t), P, w[lvl], 0, w[lvl], _p(cat), 0, 2 * w[lvl])
            K("copy_channels", _p(skips[lvl]), P, w[lvl], 0, w[lvl], _p(cat), w[lvl], 2 * w[lvl])
            h = cb.forward(K, ca.forward(K, cat, n, hh, ww), n, hh, ww)
        out = self.head.forward(K, h, n, H, W)
        K("axpy", ctypes.c_float(1.0), _p(x), _p(out), out.numel())
        return out

    def backward(self, dout):
        K, w, n = self.K, self.widths, self.n
        dh = self.head.backward(K, dout.clone())
        dskips = [None, None, None]
        for lvl in (0, 1, 2):
            cu, ca, cb = self.dec[lvl]
            hh, ww = self.sizes[lvl]
            P = n * hh * ww
            dcat = ca.backward(K, cb.backward(K, dh))
            dt = torch.empty((P, w[lvl]), device="cuda")
            ds = torch.empty((P, w[lvl]), device="cuda")
            K("copy_channels", _p(dcat), P, w[lvl], 0, 2 * w[lvl], _p(dt), 0, w[lvl])
            K("copy_channels", _p(dcat), P, w[lvl], w[lvl], 2 * w[lvl], _p(ds), 0, w[lvl])
            dskips[lvl] = ds
            dup = cu.backward(K, dt)
            dh = torch.empty((n * (hh // 2) * (ww // 2), w[lvl + 1]), device="cuda")
            K("up2_bwd", _p(dup), n, hh // 2, ww // 2, w[lvl + 1], _p(dh))
        for lvl in (3, 2, 1, 0):
            ca, cb = self.enc[lvl]
            hh, ww = self.sizes[lvl]
            if lvl < 3:   # gradient of the level's output: through the pool, plus the skip
                dfull = torch.empty((n * hh * ww, w[lvl]), device="cuda")
                K("pool2_bwd", _p(dh), n, hh, ww, w[lvl], _p(dfull))
                K("axpy", ctypes.c_float(1.0), _p(dskips[lvl]), _p(dfull), dfull.numel())
                dh = dfull
            dh = ca.backward(K, cb.backward(K, dh), need_dx=lvl > 0)

    def step(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        for layer in self.layers():
            for prm in layer.params():
                self.K("adam", _p(prm.w), _p(prm.g), _p(prm.m), _p(prm.v), prm.w.numel(), ctypes.c_float(lr),
                       ctypes.c_float(b1), ctypes.c_float(b2), ctypes.c_float(eps), self.t)

    def mse(self, out, target):
        """Loss (FP64 device scalar) and its gradient with respect to out."""
        grad = torch.empty_like(out)
        self.K("mse", _p(out), _p(target), out.numel(), _p(grad), _p(self.K.loss))
        return self.K.loss[:1], grad

    # object-level helpers: f [X][J][Q] (one object) <-> [X*J][Q]
    def predict(self, f1, scale, floor):
        """f^0 = max(scale * U(f1 / scale), floor) for one object f1 [X][J][Q]."""
        X, J, Q = f1.shape
        x = torch.empty_like(f1)
        self.K("scale_clamp", _p(f1), ctypes.c_float(1.0 / scale), ctypes.c_float(-math.inf), _p(x), x.numel())
        out = self.forward(x.view(X * J, Q), 1, X, J)
        f0 = torch.empty_like(f1)
        self.K("scale_clamp", _p(out), ctypes.c_float(scale), ctypes.c_float(floor), _p(f0), f0.numel())
        return f0

    def state(self):
        return {f"p{k}": prm.w.detach().cpu().numpy() for k, prm in
                enumerate(p for layer in self.layers() for p in layer.params())}


# ---------------------------------------------------------------------------
# training pairs from the forward model (the synthetic-input recipe)
# ---------------------------------------------------------------------------

class PairMaker:
    """Phantom -> counts y ~ Poisson(kappa A f) (peak log-uniform in [1e2, 1e4]),
    drawn on the device (caxsi_nn_poisson, key 100 + seed) -> the first EM-type
    iterate from the flat start (penalty beta = 1e-3 sum(y)/(XJQ), delta =
    0.01 f_init), with the object in count units as the target."""

    def __init__(self, plan, g, path="table_fp32"):
        self.plan, self.g = plan, g
        self.path = caxsi.PATHS[path]
        self.b1_sum = float(plan.adjoint(torch.ones((g.M, g.N), device="cuda"), path=self.path).double().sum())
        self.lib = caxsi.load()

    def counts(self, mean, kappa, key):
        """y ~ Poisson(kappa * mean) on the device (float32, integer values)."""
        y = torch.empty_like(mean)
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        caxsi._check(self.lib.caxsi_nn_poisson(_p(mean), ctypes.c_float(kappa), mean.numel(),
                                               ctypes.c_uint64(key), _p(y), s), "caxsi_nn_poisson")
        return y

    def make(self, seed, y=None, f_ref=None):
        import synth
        g = self.g
        if y is None:
            f_true = synth.phantom_torch(g, seed, "cuda")
            mean = self.plan.forward(f_true, path=self.path)
            peak = synth.log_uniform_peak(seed)
            kappa = peak / float(mean.max())
            y = self.counts(mean, kappa, 100 + seed)
            f_ref = f_true * kappa
        ysum = float(y.sum())
        f_init = ysum / self.b1_sum
        beta = 1e-3 * ysum / (g.X * g.J * g.Q)
        delta = 0.01 * f_init
        f1 = torch.full((g.X, g.J, g.Q), f_init, device="cuda")
        self.plan.recon_step(y, f1, beta=beta, delta=delta, path=self.path)
        return f1, f_ref, y, beta, delta, f_init


def _inputs(maker: PairMaker, seeds):
    """Normalised network inputs and targets of the objects `seeds`: f1 / s and
    f_ref / s with s = mean(f1), stacked as [n*X*J][Q]."""
    g = maker.g
    xs, ts = [], []
    for sd in seeds:
        f1, f_ref, *_ = maker.make(sd)
        s = float(f1.mean())
        xs.append((f1 / s).view(g.X * g.J, g.Q))
        ts.append((f_ref / s).view(g.X * g.J, g.Q))
    return torch.cat(xs).contiguous(), torch.cat(ts).contiguous()


def heldout_loss(net: UNet, maker: PairMaker, held) -> float:
    """Mean normalised MSE of the network on held-out inputs (x, t, n) from _inputs."""
    x, t, n = held
    g = maker.g
    out = net.forward(x, n, g.X, g.J)
    loss, _ = net.mse(out, t)
    return float(loss)


def train(net: UNet, maker: PairMaker, steps: int, lr: float = 1e-3, batch: int = 4, first_seed: int = 100000,
          log=None, heldout_seeds=None):
    """Adam on the normalised MSE ||U(f1/s) - f_ref/s||^2 / n with s = mean(f1) per
    object, `batch` objects per step (seeds first_seed, first_seed + 1, ...),
    cosine-decayed learning rate.  With log = L, every L steps (and at the last)
    records (step, training loss of the step's batch, mean loss on the held-out
    objects heldout_seeds, which no step trains on)."""
    g = maker.g
    held = None
    if heldout_seeds:
        hx, ht = _inputs(maker, heldout_seeds)
        held = (hx, ht, len(heldout_seeds))
    losses = []
    for k in range(steps):
        x, tgt = _inputs(maker, range(first_seed + k * batch, first_seed + (k + 1) * batch))
        out = net.forward(x, batch, g.X, g.J)
        loss, grad = net.mse(out, tgt)
        train_loss = float(loss) if log is not None else None
        net.backward(grad)
        net.step(lr * 0.5 * (1.0 + math.cos(math.pi * k / max(1, steps))))
        if log is not None and (k % log == 0 or k == steps - 1):
            losses.append((k, train_loss, heldout_loss(net, maker, held) if held else None))
    return losses


def train_step_scalings(net: UNet, maker: PairMaker, T: int = 10, samples: int = 40, lr: float = 2e-2,
                        first_seed: int = 200000):
    """Per-iteration relaxation factors s_1..s_T of the EM-type iterations that
    follow the warm start (f <- max(f + s_t (U(f) - f), floor)), learned by
    differentiating T unrolled, checkpointed iterations (autodiff.unrolled_em) of
    the normalised error ||f_T - f_ref||^2 / ||f_ref||^2 over training objects."""
    from . import autodiff
    op = autodiff.Operator(maker.plan)
    relax = torch.ones(T, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([relax], lr=lr)
    for k in range(samples):
        f1, f_ref, y, beta, delta, _ = maker.make(first_seed + k)
        s = float(f1.mean())
        with torch.no_grad():
            f0 = net.predict(f1, s, 1e-3 * s)
        out = autodiff.unrolled_em(op, y, f0, T, beta=beta, delta=delta, checkpoint=True, relax=relax,
                                   floor=1e-3 * s)
        loss = torch.sum((out.double() - f_ref.double()) ** 2) / torch.sum(f_ref.double() ** 2)
        opt.zero_grad()
        loss.backward()
        opt.step()
    return relax.detach()


def relaxed_iterations(maker: PairMaker, y, f0, relax, beta, delta, floor):
    """The EM-type iterations from f0 with step scalings `relax` (no gradients)."""
    from . import autodiff
    with torch.no_grad():
        return autodiff.unrolled_em(autodiff.Operator(maker.plan), y, f0, len(relax), beta=beta, delta=delta,
                                    checkpoint=False, relax=relax, floor=floor)
