"""FP64 CPU oracle of the variational solvers of Section 4.2 that call A and A*.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path and imports nothing from it.

Written in plain PyTorch CPU ops in float64 so that autograd of the unrolled
iterations gives the reference gradients for the differentiable solvers.  A
and A* enter as ``LinearOp`` (a torch.autograd.Function around the FP64
oracle of ``tat_oracle`` or any matrix pair), whose backward is the Euclidean
transpose: A^T = (W_X / W_Y) A* because A* = W_X^{-1} A^T W_Y with scalar
weights (Eq. innerProducts).

* ``nnls`` -- projected gradient descent for min_{f>=0} 1/2||Af - g||^2,
  Eqs. NNLS and NNLS-projstep, with the region-of-interest projection of
  Eq. projectionHalfCircle when a mask is given; f^(0) = 0.
* ``tv_pdhg`` -- primal-dual hybrid gradient (Chambolle-Pock) for
  min_{f>=0} 1/2||Af - g||^2 + alpha ||grad f||_1, Eqs. PDHG-dual,
  PDHG-primal, PDHG-relaxation.  Readings: (i) the TV term is dualised with
  the data term, K = [A; s grad_h] (s > 0 a balancing scale, TV dual bound
  alpha/s), so prox_{alpha TV} needs no inner solver; (ii) the relaxation is
  the standard extrapolation fbar = f^(k+1) + (f^(k+1) - f^(k)) (theta = 1);
  the printed form f^(k+1) + mu (f^(k) - f^(k+1)) would not extrapolate;
  (iii) positivity (Eq. minim's f >= 0) and Pi_Omega0 are applied in the
  primal step.
* ``power_norm_sq`` -- ||A||^2 = largest eigenvalue of A*A by power iteration
  (for the step sizes lambda < 2/||A||^2 and sigma tau ||K||^2 < 1).
* ``grad_h`` / ``div_h`` -- forward differences / h with zero across the last
  column and row, and div_h = -grad_h^T.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .tat_oracle import OraclePlan, adjoint, forward

_F64 = torch.float64


class _Apply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, op, transpose):
        ctx.op, ctx.transpose = op, transpose
        return op._apply(x, transpose)

    @staticmethod
    def backward(ctx, g):
        op = ctx.op
        if ctx.transpose:      # (A*)^T = (W_Y / W_X) A
            return op._apply(g, False) / op.wx_over_wy, None, None
        return op._apply(g, True) * op.wx_over_wy, None, None   # A^T = (W_X / W_Y) A*


class LinearOp:
    """A linear map A with its adjoint A* on batched torch float64 tensors.

    ``fwd`` / ``adj`` act on one numpy sample; ``wx_over_wy`` = W_X / W_Y
    (1 for a plain matrix pair).  ``A`` / ``Astar`` are differentiable.
    """

    def __init__(self, fwd, adj, x_shape, y_shape, wx_over_wy=1.0):
        self.fwd, self.adj = fwd, adj
        self.x_shape, self.y_shape = tuple(x_shape), tuple(y_shape)
        self.wx_over_wy = float(wx_over_wy)

    def _apply(self, x, transpose):
        fn, shape = (self.adj, self.y_shape) if transpose else (self.fwd, self.x_shape)
        xs = x.detach().reshape(-1, *shape).numpy()
        out = np.stack([np.asarray(fn(v), dtype=np.float64) for v in xs])
        return torch.from_numpy(out).reshape(*x.shape[: x.dim() - len(shape)], *out.shape[1:])

    def A(self, f):
        return _Apply.apply(f, self, False)

    def Astar(self, g):
        return _Apply.apply(g, self, True)


def plan_op(P: OraclePlan) -> LinearOp:
    """The oracle's A (Algorithm 1) and A* (Algorithm 2) as a LinearOp."""
    return LinearOp(lambda f: forward(P, f), lambda g: adjoint(P, g), (P.n, P.n), (P.n_det, P.n_t),
                    P.W_X / P.W_Y)


def matrix_op(M: np.ndarray, n: int) -> LinearOp:
    """A = M acting on flattened n x n images (A* = M^T, unit weights)."""
    M = np.asarray(M, dtype=np.float64)
    return LinearOp(lambda f: M @ f.reshape(-1), lambda g: (M.T @ g).reshape(n, n), (n, n), (M.shape[0],), 1.0)


# ------------------------------------------------------------------ TV pieces

def grad_h(f: torch.Tensor, h: float) -> torch.Tensor:
    """(..., n, n) -> (..., 2, n, n): forward differences / h in x (last axis) then y."""
    gx = torch.zeros_like(f)
    gy = torch.zeros_like(f)
    gx[..., :, :-1] = (f[..., :, 1:] - f[..., :, :-1]) / h
    gy[..., :-1, :] = (f[..., 1:, :] - f[..., :-1, :]) / h
    return torch.stack((gx, gy), dim=-3)


def div_h(p: torch.Tensor, h: float) -> torch.Tensor:
    """(..., 2, n, n) -> (..., n, n): div_h = -grad_h^T (backward differences / h)."""
    px, py = p[..., 0, :, :], p[..., 1, :, :]
    dx = torch.zeros_like(px)
    dy = torch.zeros_like(py)
    dx[..., :, :-1] += px[..., :, :-1]
    dx[..., :, 1:] -= px[..., :, :-1]
    dy[..., :-1, :] += py[..., :-1, :]
    dy[..., 1:, :] -= py[..., :-1, :]
    return (dx + dy) / h


def _project_ball(u: torch.Tensor, bound: float) -> torch.Tensor:
    """Pointwise projection of the (x, y) pairs of u (..., 2, n, n) onto |u| <= bound."""
    nrm = torch.sqrt(torch.clamp((u * u).sum(dim=-3, keepdim=True), min=1e-300))
    return u / torch.clamp(nrm / bound, min=1.0)


# ------------------------------------------------------------------ single steps

def pdhg_dual_data(q, Af, g, sigma):
    """Eq. PDHG-dual: prox of sigma F* for F = 1/2 ||. - g||^2."""
    return (q + sigma * (Af - g)) / (1.0 + sigma)


def tv_dual(p, fbar, sigma, alpha, s, h):
    """Dual step of the TV block of K: proj_{|p| <= alpha/s}(p + sigma s grad_h fbar)."""
    return _project_ball(p + sigma * s * grad_h(fbar, h), alpha / s)


def tv_primal(f, Asq, p, tau, s, h, mask=None):
    """Eq. PDHG-primal with K^T (q, p) = A* q - s div_h p, then positivity and Pi_Omega0;
    Eq. PDHG-relaxation with theta = 1.  Returns (f_new, fbar)."""
    f_new = torch.clamp(f - tau * (Asq - s * div_h(p, h)), min=0.0)
    if mask is not None:
        f_new = f_new * mask
    return f_new, 2.0 * f_new - f


def nnls_step(op: LinearOp, f, g, lam, mask=None):
    """Eqs. NNLS / NNLS-projstep (projectionHalfCircle with a mask)."""
    f_half = f - lam * op.Astar(op.A(f) - g)
    f_new = torch.clamp(f_half, min=0.0)
    return f_new * mask if mask is not None else f_new


# ------------------------------------------------------------------ solvers

def power_norm_sq(op: LinearOp, v0: torch.Tensor, iters: int) -> float:
    """Largest eigenvalue of A*A (= ||A||^2 in the weighted norms) by power iteration."""
    v = v0 / torch.linalg.vector_norm(v0)
    est = 0.0
    with torch.no_grad():
        for _ in range(iters):
            w = op.Astar(op.A(v))
            est = float((w * v).sum())
            v = w / torch.linalg.vector_norm(w)
    return est


def nnls(op: LinearOp, g, lam, iters, mask=None, f0=None):
    """iters steps of projected gradient from f^(0) = 0 (or f0)."""
    f = torch.zeros(*g.shape[: g.dim() - len(op.y_shape)], *op.x_shape, dtype=_F64) if f0 is None else f0
    for _ in range(iters):
        f = nnls_step(op, f, g, lam, mask)
    return f


def pdhg_steps(norm_sq: float, h: float, safety: float = 0.99):
    """Balanced step sizes for K = [A; s grad_h]: s^2 ||grad_h||^2 <= s^2 8/h^2 = ||A||^2,
    so ||K||^2 <= 2 ||A||^2, and sigma = tau = safety / sqrt(2 ||A||^2)."""
    s = math.sqrt(norm_sq) * h / math.sqrt(8.0)
    step = safety / math.sqrt(2.0 * norm_sq)
    return step, step, s


def tv_pdhg(op: LinearOp, g, alpha, h, iters, sigma, tau, s, mask=None):
    """iters PDHG iterations from f^(0) = 0, q^(0) = 0, p^(0) = 0."""
    batch = g.shape[: g.dim() - len(op.y_shape)]
    f = torch.zeros(*batch, *op.x_shape, dtype=_F64)
    fbar = f
    q = torch.zeros_like(g)
    p = torch.zeros(*batch, 2, *op.x_shape, dtype=_F64)
    for _ in range(iters):
        q = pdhg_dual_data(q, op.A(fbar), g, sigma)
        p = tv_dual(p, fbar, sigma, alpha, s, h)
        f, fbar = tv_primal(f, op.Astar(q), p, tau, s, h, mask)
    return f


def tv_objective(op: LinearOp, f, g, alpha, h, w_y=1.0, w_x=1.0):
    """1/2 W_Y ||Af - g||^2 + alpha W_X sum |grad_h f| per sample (a torch scalar per batch entry)."""
    r = op.A(f) - g
    gr = grad_h(f, h)
    tv = torch.sqrt((gr * gr).sum(dim=-3)).flatten(-2).sum(-1)
    return 0.5 * w_y * (r * r).flatten(r.dim() - len(op.y_shape)).sum(-1) + alpha * w_x * tv
