"""Batched NNLS and TV-regularised least squares on libtat's A and A* (Section 4.2).

Problem: min_{f >= 0, f = Pi_Omega0 f} 1/2 ||A f - g||^2 + alpha ||grad f||_1
(Eq. minim with the fidelity halved as in Eq. PDHG-dual; alpha = 0 is NNLS).

* NNLS: projected gradient f <- Pi_Omega0 max(0, f - lambda A*(A f - g)),
  f^(0) = 0 (Eqs. NNLS, NNLS-projstep, projectionHalfCircle); the paper leaves
  lambda open, the default is 1/||A||^2 (< 2/||A||^2 for convergence).
* TV: Chambolle-Pock primal-dual iteration with K = [A; s grad_h] (the TV
  term dualised, so no inner prox iterations) and the theta = 1
  extrapolation (Eqs. PDHG-dual, PDHG-primal, PDHG-relaxation); default
  s = ||A|| h / sqrt(8) balances the two blocks, sigma = tau = 0.99 /
  sqrt(2 ||A||^2) gives sigma tau ||K||^2 < 1.

Two paths run the same iteration:
* ``TatSolver`` -- the fast path: static device buffers, in-place fused
  element-wise kernels (include/tat_solvers.h) between the A / A* launches,
  optionally one CUDA graph per iteration replayed ``iters`` times.
* ``nnls_unrolled`` / ``tv_unrolled`` -- differentiable: every step is a
  torch.autograd.Function whose forward and backward are libtat kernels, so
  gradients flow through the unrolled iterations to g (or to anything g
  depends on).
"""
from __future__ import annotations

import math

import torch

from . import autograd as AG
from . import binding as B

_NEG_INF = -math.inf


def power_norm_sq(op, iters: int = 40, seed: int = 0) -> float:
    """||A||^2 (largest eigenvalue of A*A) by power iteration on one image.

    The start vector comes from torch's seeded generator; the few scalar
    reductions are torch's.  Returns the Rayleigh quotient of the last step
    (a lower bound that converges from below)."""
    gen = torch.Generator(device=op.device).manual_seed(seed)
    v = torch.rand((op.n, op.n), generator=gen, device=op.device, dtype=torch.float32) - 0.5
    v /= torch.linalg.vector_norm(v)
    est = torch.zeros((), device=op.device)
    for _ in range(iters):
        w = op.adjoint(op.forward(v))
        est = (w * v).sum()
        v = w / torch.linalg.vector_norm(w)
    return float(est)


def pdhg_steps(norm_sq: float, h: float, safety: float = 0.99):
    """(sigma, tau, s) for K = [A; s grad_h]: s^2 * 8/h^2 = ||A||^2 bounds ||K||^2 by 2||A||^2."""
    s = math.sqrt(norm_sq) * h / math.sqrt(8.0)
    step = safety / math.sqrt(2.0 * norm_sq)
    return step, step, s


class TatSolver:
    """Batched projected-gradient NNLS and TV-PDHG with fused element-wise steps.

    op: a ``TatOperator``; batch: number of images solved together; mask: an
    (n, n) float32 0/1 tensor (Pi_Omega0) or None.  ``h`` is the image grid
    spacing used by grad_h (default: the plan's, in units of R).
    """

    def __init__(self, op, batch: int, mask: torch.Tensor | None = None, h: float | None = None):
        self.op, self.batch = op, batch
        n, nd, nt, dev = op.n, op.n_det, op.n_t, op.device
        self.h = h if h is not None else op.info["h"] * op.desc.R
        self.mask = None
        if mask is not None:
            self.mask = mask.to(device=dev, dtype=torch.float32).contiguous()
            if self.mask.shape != (n, n):
                raise ValueError(f"mask must be ({n}, {n})")
        img = dict(dtype=torch.float32, device=dev)
        self.g = torch.zeros((batch, nd, nt), **img)       # data (static for graphs)
        self.f = torch.zeros((batch, n, n), **img)         # primal iterate
        self.fbar = torch.zeros((batch, n, n), **img)      # extrapolated primal (PDHG)
        self.x_tmp = torch.zeros((batch, n, n), **img)     # A*(...) result
        self.y_tmp = torch.zeros((batch, nd, nt), **img)   # A(...) result / residual
        self.q = torch.zeros((batch, nd, nt), **img)       # data dual (PDHG)
        self.p = torch.zeros((batch, 2, n, n), **img)      # TV dual (PDHG)
        op.workspace(batch)                                 # allocate before any capture
        self.nx, self.ny = batch * n * n, batch * nd * nt
        self._graphs = {}

    def _s(self):
        return torch.cuda.current_stream(self.op.device).cuda_stream

    # ---------------------------------------------------------------- one iteration each

    def _nnls_iter(self, lam: float):
        op, st = self.op, self._s()
        op.forward(self.f, out=self.y_tmp)                                     # A f
        B.tat_axpby_clamp(self.ny, 1.0, self.y_tmp.data_ptr(), -1.0, self.g.data_ptr(), _NEG_INF, 0, 1,
                          self.y_tmp.data_ptr(), st)                           # r = A f - g
        op.adjoint(self.y_tmp, out=self.x_tmp)                                 # A* r
        B.tat_axpby_clamp(self.nx, 1.0, self.f.data_ptr(), -lam, self.x_tmp.data_ptr(), 0.0, _p(self.mask),
                          self.op.n * self.op.n, self.f.data_ptr(), st)        # f = P max(0, f - lam A* r)

    def _tv_iter(self, alpha: float, sigma: float, tau: float, s: float):
        op, st, n = self.op, self._s(), self.op.n
        h_eff = self.h / s
        op.forward(self.fbar, out=self.y_tmp)                                  # A fbar
        B.tat_pd_dual_data(self.ny, sigma, self.y_tmp.data_ptr(), self.g.data_ptr(), self.q.data_ptr(),
                           self.q.data_ptr(), st)
        B.tat_tv_dual(self.batch, n, h_eff, sigma, alpha / s, self.fbar.data_ptr(), self.p.data_ptr(),
                      self.p.data_ptr(), st)
        op.adjoint(self.q, out=self.x_tmp)                                     # A* q
        B.tat_tv_primal(self.batch, n, h_eff, tau, self.x_tmp.data_ptr(), self.p.data_ptr(), _p(self.mask),
                        self.f.data_ptr(), self.f.data_ptr(), self.fbar.data_ptr(), st)

    # ---------------------------------------------------------------- drivers

    def _graph(self, key, body):
        """One CUDA graph per (method, parameters) holding one iteration.

        Warm-up runs the iteration once on the live state; callers reset the
        state after this returns."""
        G = self._graphs.get(key)
        if G is None:
            dev = self.op.device
            side = torch.cuda.Stream(dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(side):
                body()
            torch.cuda.current_stream(dev).wait_stream(side)
            G = torch.cuda.CUDAGraph()
            with torch.cuda.graph(G):
                body()
            if len(self._graphs) >= 4:
                self._graphs.clear()
            self._graphs[key] = G
        return G

    def _iterate(self, key, body, iters: int, graph: bool, state):
        G = self._graph(key, body) if graph else None
        for t in state:
            t.zero_()
        for _ in range(iters):
            if G is not None:
                G.replay()
            else:
                body()

    def _load(self, g: torch.Tensor):
        if tuple(g.shape) != tuple(self.g.shape):
            raise ValueError(f"g must have shape {tuple(self.g.shape)}")
        self.g.copy_(g)

    def nnls(self, g: torch.Tensor, iters: int, lam: float, graph: bool = False) -> torch.Tensor:
        """iters projected-gradient steps from f = 0; returns the (B, n, n) iterate (the solver's state)."""
        if not lam > 0:
            raise ValueError("lam must be positive")
        self._load(g)
        self._iterate(("nnls", lam), lambda: self._nnls_iter(lam), iters, graph, (self.f,))
        return self.f

    def tv(self, g: torch.Tensor, alpha: float, iters: int, sigma: float, tau: float, s: float,
           graph: bool = False) -> torch.Tensor:
        """iters PDHG iterations from f = fbar = q = p = 0; returns the (B, n, n) iterate."""
        if not (alpha > 0 and sigma > 0 and tau > 0 and s > 0):
            raise ValueError("alpha, sigma, tau and s must be positive")
        self._load(g)
        self._iterate(("tv", alpha, sigma, tau, s), lambda: self._tv_iter(alpha, sigma, tau, s), iters, graph,
                      (self.f, self.fbar, self.q, self.p))
        return self.f


def _p(t):
    return 0 if t is None else t.data_ptr()


# ------------------------------------------------------------------ differentiable

def nnls_unrolled(op, g: torch.Tensor, iters: int, lam: float, mask: torch.Tensor | None = None) -> torch.Tensor:
    """The NNLS iteration as a differentiable function of g (batch (B, n_det, n_t) or one sinogram)."""
    f = torch.zeros((*g.shape[:-2], op.n, op.n), dtype=torch.float32, device=g.device)
    for _ in range(iters):
        r = AG.AxpbyClampFn.apply(AG.A(op, f), g, 1.0, -1.0, _NEG_INF, None)
        f = AG.AxpbyClampFn.apply(f, AG.Astar(op, r), 1.0, -lam, 0.0, mask)
    return f


def tv_unrolled(op, g: torch.Tensor, alpha: float, iters: int, sigma: float, tau: float, s: float,
                mask: torch.Tensor | None = None, h: float | None = None) -> torch.Tensor:
    """The TV-PDHG iteration as a differentiable function of g."""
    h = h if h is not None else op.info["h"] * op.desc.R
    h_eff = h / s
    batch = g.shape[:-2]
    f = torch.zeros((*batch, op.n, op.n), dtype=torch.float32, device=g.device)
    fbar = f
    q = torch.zeros_like(g)
    p = torch.zeros((*batch, 2, op.n, op.n), dtype=torch.float32, device=g.device)
    for _ in range(iters):
        q = AG.PdDualDataFn.apply(q, AG.A(op, fbar), g, sigma)
        p = AG.TvDualFn.apply(p, fbar, sigma, alpha / s, h_eff)
        f, fbar = AG.TvPrimalFn.apply(f, AG.Astar(op, q), p, tau, h_eff, mask)
    return f
