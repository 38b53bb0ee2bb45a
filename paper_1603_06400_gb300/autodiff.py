"""Automatic differentiation over the scatter operators.

A and A^T are torch.autograd functions, each the other's backward (A is linear,
so the vector-Jacobian product of A is A^T).  The EM update of Eq. 10 has its
own reverse-mode kernel (caxsi_em_update_vjp).  On top of these sits the
reconstruction unrolled over a fixed number of iterations, optionally
checkpointed per iteration (activations are recomputed in the backward pass
instead of being kept), and differentiable with respect to its start and to
per-iteration step scalings.  Operators and updates run in the library's
kernels through the C ABI, the likelihood ratio y / (A f + r) and its reverse
mode included (caxsi_ratio, caxsi_ratio_vjp); only the losses are torch glue.
A single object is f [X, J, Q]; a batch is f [nb, X, J, Q] with y [nb, M, N],
each object a voxel range of the shared geometry; objects of different
geometries (MultiOperator over a caxsi.Multi set) are packed flat arrays.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint as _checkpoint

from . import caxsi


class Operator:
    """y = A f with autograd.  `ranges` ([nb, 2] voxel ranges) applies to batches."""

    def __init__(self, plan: "caxsi.Plan", path: str = "table_fp32", ranges=None):
        self.plan = plan
        self.path = caxsi.PATHS[path]
        self.ranges = ranges

    # raw calls (no autograd)
    def _fwd(self, f):
        if f.dim() == 4:
            return self.plan.forward_batch(f, ranges=self.ranges, path=self.path)
        return self.plan.forward(f, path=self.path)

    def _adj(self, w):
        if w.dim() == 3:
            return self.plan.adjoint_batch(w, ranges=self.ranges, path=self.path)
        return self.plan.adjoint(w, path=self.path)

    def __call__(self, f):
        return _Forward.apply(f.contiguous(), self)

    def T(self, w):
        return _Adjoint.apply(w.contiguous(), self)

    def update(self, f, b1, b2, beta=0.0, delta=0.0):
        return _Update.apply(f.contiguous(), b1.contiguous(), b2.contiguous(), self, float(beta), float(delta))

    def _em_update(self, f, b1, b2, beta, delta):
        return self.plan.em_update(f, b1, b2, beta, delta)

    def _em_update_vjp(self, f, b1, b2, g, beta, delta):
        return self.plan.em_update_vjp(f, b1, b2, g, beta, delta)

    def ratio(self, g, y, r=None):
        """y / (g + r) (0 where g + r <= 0), differentiable with respect to g."""
        return _Ratio.apply(g.contiguous(), y.contiguous(), None if r is None else r.contiguous(), self)


class MultiOperator:
    """The operator of a caxsi.Multi set (objects of different geometries, packed
    flat arrays) with the interface of Operator, so that em_step and unrolled_em
    run on it: A, A^T and the update each one launch for all objects."""

    def __init__(self, multi: "caxsi.Multi"):
        self.multi = multi
        self.plan = multi.plans[0]      # the ratio kernel's device and error word
        self.path = caxsi.PATH_DIRECT

    def _fwd(self, f):
        return self.multi.forward(f, path=self.path)

    def _adj(self, w):
        return self.multi.adjoint(w, path=self.path)

    __call__ = Operator.__call__
    T = Operator.T
    ratio = Operator.ratio

    def update(self, f, b1, b2, beta=0.0, delta=0.0):
        return _Update.apply(f.contiguous(), b1.contiguous(), b2.contiguous(), self, float(beta), float(delta))

    def _em_update(self, f, b1, b2, beta, delta):
        return self.multi.em_update(f, b1, b2, beta, delta)

    def _em_update_vjp(self, f, b1, b2, g, beta, delta):
        return self.multi.em_update_vjp(f, b1, b2, g, beta, delta)


class _Forward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, op):
        ctx.op = op
        return op._fwd(f)

    @staticmethod
    def backward(ctx, g):
        return ctx.op._adj(g.contiguous()), None


class _Adjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, op):
        ctx.op = op
        return op._adj(w)

    @staticmethod
    def backward(ctx, g):
        return ctx.op._fwd(g.contiguous()), None


class _Update(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, b1, b2, op, beta, delta):
        ctx.save_for_backward(f, b1, b2)
        ctx.op, ctx.beta, ctx.delta = op, beta, delta
        return op._em_update(f, b1, b2, beta, delta)

    @staticmethod
    def backward(ctx, g):
        f, b1, b2 = ctx.saved_tensors
        gf, gb2 = ctx.op._em_update_vjp(f, b1, b2, g.contiguous(), ctx.beta, ctx.delta)
        return gf, None, gb2, None, None, None


class _Ratio(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, y, r, op):
        ctx.save_for_backward(g, y, r)
        ctx.op = op
        return op.plan.ratio(g, y, r)

    @staticmethod
    def backward(ctx, grad):
        g, y, r = ctx.saved_tensors
        return ctx.op.plan.ratio_vjp(g, y, grad.contiguous(), r), None, None, None


def em_step(op: Operator, y, f, b1, r=None, beta=0.0, delta=0.0):
    """One EM-type iteration (Algorithm 4): z = A f + r, b2 = A^T (y / z), Eq. 10."""
    return op.update(f, b1, op.T(op.ratio(op(f), y, r)), beta, delta)


def unrolled_em(op: Operator, y, f0, n_iter: int = 10, r=None, beta=0.0, delta=0.0,
                checkpoint: bool = True, relax=None, floor=None):
    """n_iter EM-type iterations from f0, differentiable with respect to f0 and to
    `relax` (optional per-iteration step scalings s_t: f <- f + s_t (U(f) - f),
    then max(f, floor) when floor is given, so that f stays positive).
    With checkpoint=True each iteration keeps only its input for the backward
    pass and recomputes the rest."""
    with torch.no_grad():
        b1 = op.T(torch.ones_like(y))
    f = f0
    for t in range(n_iter):
        def step(fc, t=t):
            fn = em_step(op, y, fc, b1, r, beta, delta)
            if relax is not None:
                fn = fc + relax[t] * (fn - fc)
                if floor is not None:
                    fn = torch.clamp(fn, min=floor)
            return fn
        f = _checkpoint(step, f, use_reentrant=False) if checkpoint else step(f)
    return f
