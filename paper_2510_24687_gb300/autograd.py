"""torch.autograd Functions over libtat's kernels: A, A* and the fused solver steps.

Every forward and backward here launches libtat kernels (include/tat.h,
include/tat_solvers.h); torch only allocates the outputs.

Backward of the operators (Eq. innerProducts): libtat's A* is the adjoint in
the weighted inner products, A* = W_X^{-1} A^T W_Y with scalar weights, so
the Euclidean transposes that autograd needs are
    A^T     = (W_X / W_Y) A*      (backward of A)
    (A*)^T  = (W_Y / W_X) A       (backward of A*).
"""
from __future__ import annotations

import math

import torch

from . import binding as B

_NEG_INF = -math.inf


def _stream(t: torch.Tensor) -> int:
    return torch.cuda.current_stream(t.device).cuda_stream


def _c(t):
    return t if t is None or t.is_contiguous() else t.contiguous()


def _p(t):
    return 0 if t is None else t.data_ptr()


def scale_(t: torch.Tensor, a: float) -> torch.Tensor:
    """t *= a in place (one libtat launch)."""
    B.tat_axpby_clamp(t.numel(), a, t.data_ptr(), 0.0, 0, _NEG_INF, 0, 1, t.data_ptr(), _stream(t))
    return t


def _check_image_batch(x: torch.Tensor, n: int) -> int:
    if x.dtype != torch.float32 or not x.is_cuda or x.shape[-1] != n or x.shape[-2] != n:
        raise ValueError(f"expected a float32 CUDA tensor of shape (..., {n}, {n})")
    return x.numel() // (n * n)


class TatForwardFn(torch.autograd.Function):
    """g = A f (Algorithm 1); backward: grad_f = (W_X / W_Y) A* grad_g."""

    @staticmethod
    def forward(ctx, f, op):
        ctx.op = op
        return op.forward(_c(f))

    @staticmethod
    def backward(ctx, grad_g):
        op = ctx.op
        return scale_(op.adjoint(_c(grad_g)), op.W_X / op.W_Y), None


class TatAdjointFn(torch.autograd.Function):
    """f = A* g (Algorithm 2); backward: grad_g = (W_Y / W_X) A grad_f."""

    @staticmethod
    def forward(ctx, g, op):
        ctx.op = op
        return op.adjoint(_c(g))

    @staticmethod
    def backward(ctx, grad_f):
        op = ctx.op
        return scale_(op.forward(_c(grad_f)), op.W_Y / op.W_X), None


def A(op, f):
    """Differentiable A f."""
    return TatForwardFn.apply(f, op)


def Astar(op, g):
    """Differentiable A* g."""
    return TatAdjointFn.apply(g, op)


class AxpbyClampFn(torch.autograd.Function):
    """out = mask * max(lo, a x + b y); mask (n x n) repeats over the leading dimensions."""

    @staticmethod
    def forward(ctx, x, y, a, b, lo, mask):
        x, y = _c(x), _c(y)
        out = torch.empty_like(x)
        period = mask.numel() if mask is not None else 1
        B.tat_axpby_clamp(x.numel(), a, x.data_ptr(), b, _p(y), lo, _p(mask), period, out.data_ptr(), _stream(x))
        ctx.save_for_backward(out)
        ctx.a, ctx.b, ctx.lo, ctx.mask, ctx.period, ctx.has_y = a, b, lo, mask, period, y is not None
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (out,) = ctx.saved_tensors
        grad_out = _c(grad_out)
        gx = torch.empty_like(out) if ctx.needs_input_grad[0] else None
        gy = torch.empty_like(out) if ctx.has_y and ctx.needs_input_grad[1] else None
        if gx is not None or gy is not None:
            B.tat_axpby_clamp_backward(out.numel(), out.data_ptr(), ctx.lo, _p(ctx.mask), ctx.period,
                                       grad_out.data_ptr(), ctx.a, _p(gx), ctx.b, _p(gy), _stream(out))
        return gx, gy, None, None, None, None


class PdDualDataFn(torch.autograd.Function):
    """q_new = (q + sigma (Af - g)) / (1 + sigma) (Eq. PDHG-dual)."""

    @staticmethod
    def forward(ctx, q, Af, g, sigma):
        q, Af, g = _c(q), _c(Af), _c(g)
        out = torch.empty_like(q)
        B.tat_pd_dual_data(q.numel(), sigma, Af.data_ptr(), g.data_ptr(), q.data_ptr(), out.data_ptr(), _stream(q))
        ctx.sigma = sigma
        return out

    @staticmethod
    def backward(ctx, G):
        G = _c(G)
        s = ctx.sigma
        grads = []
        for need, coef in zip(ctx.needs_input_grad[:3], (1.0 / (1.0 + s), s / (1.0 + s), -s / (1.0 + s))):
            if need:
                out = torch.empty_like(G)
                B.tat_axpby_clamp(G.numel(), coef, G.data_ptr(), 0.0, 0, _NEG_INF, 0, 1, out.data_ptr(), _stream(G))
                grads.append(out)
            else:
                grads.append(None)
        return (*grads, None)


class TvDualFn(torch.autograd.Function):
    """p_new = proj_{|p| <= bound}(p + sigma grad_h fbar) with h = h_eff; p is (..., 2, n, n)."""

    @staticmethod
    def forward(ctx, p, fbar, sigma, bound, h_eff):
        p, fbar = _c(p), _c(fbar)
        n = fbar.shape[-1]
        batch = _check_image_batch(fbar, n)
        out = torch.empty_like(p)
        B.tat_tv_dual(batch, n, h_eff, sigma, bound, fbar.data_ptr(), p.data_ptr(), out.data_ptr(), _stream(p))
        ctx.save_for_backward(p, fbar)
        ctx.args = (batch, n, h_eff, sigma, bound)
        return out

    @staticmethod
    def backward(ctx, G):
        p, fbar = ctx.saved_tensors
        batch, n, h_eff, sigma, bound = ctx.args
        G = _c(G)
        gp = torch.empty_like(p)
        gf = torch.empty_like(fbar) if ctx.needs_input_grad[1] else None
        B.tat_tv_dual_backward(batch, n, h_eff, sigma, bound, fbar.data_ptr(), p.data_ptr(), G.data_ptr(),
                               gp.data_ptr(), _p(gf), _stream(p))
        return (gp if ctx.needs_input_grad[0] else None), gf, None, None, None


class TvPrimalFn(torch.autograd.Function):
    """(f_new, fbar) with f_new = mask max(0, f - tau (Asq - div_h p)), fbar = 2 f_new - f."""

    @staticmethod
    def forward(ctx, f, Asq, p, tau, h_eff, mask):
        f, Asq, p = _c(f), _c(Asq), _c(p)
        n = f.shape[-1]
        batch = _check_image_batch(f, n)
        f_new, fbar = torch.empty_like(f), torch.empty_like(f)
        B.tat_tv_primal(batch, n, h_eff, tau, Asq.data_ptr(), p.data_ptr(), _p(mask), f.data_ptr(), f_new.data_ptr(),
                        fbar.data_ptr(), _stream(f))
        ctx.set_materialize_grads(False)
        ctx.save_for_backward(f_new)
        ctx.args = (batch, n, h_eff, tau)
        ctx.mask = mask
        ctx.p_shape = p.shape
        return f_new, fbar

    @staticmethod
    def backward(ctx, g_fnew, g_fbar):
        (f_new,) = ctx.saved_tensors
        batch, n, h_eff, tau = ctx.args
        if g_fnew is None and g_fbar is None:
            return None, None, None, None, None, None
        g_fnew, g_fbar = _c(g_fnew), _c(g_fbar)
        need = ctx.needs_input_grad
        gf = torch.empty_like(f_new) if need[0] else None
        gA = torch.empty_like(f_new) if need[1] else None
        gp = f_new.new_empty(ctx.p_shape) if need[2] else None
        B.tat_tv_primal_backward(batch, n, h_eff, tau, f_new.data_ptr(), _p(ctx.mask), _p(g_fnew), _p(g_fbar), _p(gf),
                                 _p(gA), _p(gp), _stream(f_new))
        return gf, gA, gp, None, None, None
