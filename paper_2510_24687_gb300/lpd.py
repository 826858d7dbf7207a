"""Learned primal-dual reconstruction (Section 4.2.1, Eqs. LPD_dual, LPD_primal,
emp_loss) on libtat's operators and convolution kernels.

    q_{k+1} = q_k + Gamma(q_k, A f_k, y),    f_{k+1} = f_k + Lambda(f_k, A* q_{k+1}),
    k = 0..K-1 from f_0 = 0, q_0 = 0, with the same Gamma and Lambda in every
    iteration (weight sharing); the reconstruction is f_K.

Gamma and Lambda are each three 3x3 convolutions (in -> 32 channels, 32 -> 32,
32 -> 1; ReLU after the first two), BF16 operands with FP32 accumulation
(include/tat_lpd.h).  Training minimises the mean squared error of f_K
(Eq. emp_loss) with Adam.

The backward pass is written out by hand, in reverse iteration order, so that
every step -- the transposed convolutions, the weight gradients (accumulated
over the weight-shared iterations), the operator transposes
A^T = (W_X/W_Y) A* and (A*)^T = (W_Y/W_X) A, the loss and the optimizer --
runs in libtat kernels and the whole training step can be captured as one CUDA
graph.  Parameters live in one flat FP32 buffer (with a BF16 copy of it for the
convolutions); see ``param_layout`` for the order.
"""
from __future__ import annotations

import math

import torch

from . import binding as B

C = 32


def param_layout(cin):
    """(name, count) of one net's parameters in the flat buffer, in order; every
    entry starts at a multiple of 8 elements."""
    return [("w_in", 9 * cin * C), ("b_in", C), ("w_mid", 9 * C * C), ("b_mid", C), ("w_out", 9 * C), ("b_out", 1)]


def _offsets():
    off, table = 0, {}
    for net, cin in (("dual", 3), ("primal", 2)):
        for name, cnt in param_layout(cin):
            table[(net, name)] = (off, cnt)
            off += (cnt + 7) // 8 * 8
    return table, off


OFFSETS, NPARAM = _offsets()


def init_params(seed=0):
    """FP32 initial parameters (CPU): He-normal weights for the in and mid layers,
    zero biases, zero out layers (each block starts as the identity on q and f)."""
    g = torch.Generator().manual_seed(seed)
    p = torch.zeros(NPARAM, dtype=torch.float32)
    for net, cin in (("dual", 3), ("primal", 2)):
        for name, fan in (("w_in", 9 * cin), ("w_mid", 9 * C)):
            off, cnt = OFFSETS[(net, name)]
            p[off:off + cnt] = torch.randn(cnt, generator=g) * math.sqrt(2.0 / fan)
    return p


class LPD:
    """K-iteration learned primal-dual on one TatOperator for batches of `batch` data sets."""

    def __init__(self, op, batch, K=10, params=None, seed=0, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, autotune=True):
        self.op, self.B, self.K = op, batch, K
        # the operator's launch shapes tuned once for this batch (small images leave the
        # default column strips with too few CTAs per SM)
        self.tuned = op.autotune(batch) if autotune else None
        self.lr, self.betas, self.eps = lr, betas, eps
        dev = op.device
        self.dev = dev
        n, nd, nt = op.n, op.n_det, op.n_t
        f32 = dict(dtype=torch.float32, device=dev)
        bf = dict(dtype=torch.int16, device=dev)
        self.params = (params if params is not None else init_params(seed)).to(**f32).contiguous()
        self.wbf = torch.empty(NPARAM, **bf)
        B.tat_to_bf16(NPARAM, self.params.data_ptr(), self.wbf.data_ptr(), self._s())
        self.grad = torch.zeros(NPARAM, **f32)
        self.m = torch.zeros(NPARAM, **f32)
        self.v = torch.zeros(NPARAM, **f32)
        self.t = 0
        Bn = batch
        self.y = torch.zeros((Bn, nd, nt), **f32)
        self.f_true = torch.zeros((Bn, n, n), **f32)
        self.f = [torch.zeros((Bn, n, n), **f32) for _ in range(K + 1)]
        self.q = [torch.zeros((Bn, nd, nt), **f32) for _ in range(K + 1)]
        self.Af = [torch.empty((Bn, nd, nt), **f32) for _ in range(K)]
        self.Aq = [torch.empty((Bn, n, n), **f32) for _ in range(K)]
        self.h1d = [torch.empty((Bn, nd, nt, C), **bf) for _ in range(K)]
        self.h2d = [torch.empty((Bn, nd, nt, C), **bf) for _ in range(K)]
        self.h1p = [torch.empty((Bn, n, n, C), **bf) for _ in range(K)]
        self.h2p = [torch.empty((Bn, n, n, C), **bf) for _ in range(K)]
        # backward scratch
        self.gf = torch.empty((Bn, n, n), **f32)
        self.gq = torch.empty((Bn, nd, nt), **f32)
        self.gAf = torch.empty((Bn, nd, nt), **f32)
        self.gAq = torch.empty((Bn, n, n), **f32)
        self.tmp_x = torch.empty((Bn, n, n), **f32)
        self.tmp_y = torch.empty((Bn, nd, nt), **f32)
        self.g_h2d = torch.empty((Bn, nd, nt, C), **bf)
        self.g_h1d = torch.empty((Bn, nd, nt, C), **bf)
        self.g_h2p = torch.empty((Bn, n, n, C), **bf)
        self.g_h1p = torch.empty((Bn, n, n, C), **bf)
        self.loss = torch.zeros(1, **f32)
        sc = max(B.tat_lpd_scratch_floats(Bn, nd, nt), B.tat_lpd_scratch_floats(Bn, n, n))
        self.scratch_floats = sc
        self.scratch = torch.empty(sc, **f32)
        op.workspace(Bn)
        self.ws = op.workspace(Bn)
        self._graph = None

    # ---------------------------------------------------------------- helpers

    def _s(self):
        return torch.cuda.current_stream(self.dev).cuda_stream

    def _w(self, net, name):
        off, _ = OFFSETS[(net, name)]
        return self.wbf.data_ptr() + 2 * off

    def _p(self, net, name):
        off, _ = OFFSETS[(net, name)]
        return self.params.data_ptr() + 4 * off

    def _g(self, net, name):
        off, _ = OFFSETS[(net, name)]
        return self.grad.data_ptr() + 4 * off

    def _A(self, x, out):
        n, nd, nt = self.op.n, self.op.n_det, self.op.n_t
        B.tat_forward_batched(self.op.plan, self.B, x.data_ptr(), n * n, out.data_ptr(), nd * nt, self.ws.data_ptr(),
                              self._s())

    def _Astar(self, g, out):
        n, nd, nt = self.op.n, self.op.n_det, self.op.n_t
        B.tat_adjoint_batched(self.op.plan, self.B, g.data_ptr(), nd * nt, out.data_ptr(), n * n, self.ws.data_ptr(),
                              self._s())

    # ---------------------------------------------------------------- forward

    def _forward(self):
        s = self._s()
        n, nd, nt, Bn = self.op.n, self.op.n_det, self.op.n_t, self.B
        for k in range(self.K):
            self._A(self.f[k], self.Af[k])
            B.tat_conv_in_fwd(Bn, nd, nt, 3, self.q[k].data_ptr(), self.Af[k].data_ptr(), self.y.data_ptr(),
                              self._w("dual", "w_in"), self._p("dual", "b_in"), self.h1d[k].data_ptr(), s)
            B.tat_conv_mid_fwd(Bn, nd, nt, self.h1d[k].data_ptr(), self._w("dual", "w_mid"), self._p("dual", "b_mid"),
                               self.h2d[k].data_ptr(), s)
            B.tat_conv_out_fwd(Bn, nd, nt, self.h2d[k].data_ptr(), self._w("dual", "w_out"), self._p("dual", "b_out"),
                               self.q[k].data_ptr(), self.q[k + 1].data_ptr(), s)
            self._Astar(self.q[k + 1], self.Aq[k])
            B.tat_conv_in_fwd(Bn, n, n, 2, self.f[k].data_ptr(), self.Aq[k].data_ptr(), 0,
                              self._w("primal", "w_in"), self._p("primal", "b_in"), self.h1p[k].data_ptr(), s)
            B.tat_conv_mid_fwd(Bn, n, n, self.h1p[k].data_ptr(), self._w("primal", "w_mid"),
                               self._p("primal", "b_mid"), self.h2p[k].data_ptr(), s)
            B.tat_conv_out_fwd(Bn, n, n, self.h2p[k].data_ptr(), self._w("primal", "w_out"),
                               self._p("primal", "b_out"), self.f[k].data_ptr(), self.f[k + 1].data_ptr(), s)

    def reconstruct(self, y):
        """f_K for data y (B, n_det, n_t); returns the solver's f_K buffer."""
        self.y.copy_(y)
        self._forward()
        return self.f[self.K]

    # ---------------------------------------------------------------- backward

    def _net_backward(self, net, H, W, cin, g_out, h1, h2, g_h2, g_h1, x0, x1, x2, gx0, gx1, acc_mask):
        s = self._s()
        Bn, sc, nsc = self.B, self.scratch.data_ptr(), self.scratch_floats
        # each gradient leaves its kernel already masked by the ReLU of the layer below it
        # (g_h2 by h2 > 0, g_h1 by h1 > 0), so the next kernel reads no mask
        B.tat_conv_out_bwd(Bn, H, W, g_out.data_ptr(), h2.data_ptr(), self._w(net, "w_out"), 1, g_h2.data_ptr(), sc,
                           nsc, self._g(net, "w_out"), self._g(net, "b_out"), s)
        B.tat_conv_mid_bwd_weights(Bn, H, W, h1.data_ptr(), g_h2.data_ptr(), 0, sc, nsc, self._g(net, "w_mid"),
                                   self._g(net, "b_mid"), s)
        B.tat_conv_mid_bwd_data(Bn, H, W, g_h2.data_ptr(), 0, self._w(net, "w_mid"), h1.data_ptr(), g_h1.data_ptr(), s)
        B.tat_conv_in_bwd(Bn, H, W, cin, x0.data_ptr(), x1.data_ptr(), x2.data_ptr() if x2 is not None else 0,
                          g_h1.data_ptr(), 0, self._w(net, "w_in"), gx0.data_ptr(), gx1.data_ptr(), 0,
                          acc_mask, sc, nsc, self._g(net, "w_in"), self._g(net, "b_in"), s)

    def _backward(self):
        """Gradient of the loss w.r.t. all parameters into self.grad (zeroed first)."""
        s = self._s()
        n, nd, nt, Bn, K = self.op.n, self.op.n_det, self.op.n_t, self.B, self.K
        op = self.op
        B.tat_fill(NPARAM, 0.0, self.grad.data_ptr(), s)
        B.tat_fill(1, 0.0, self.loss.data_ptr(), s)
        cnt = Bn * n * n
        B.tat_mse(cnt, self.f[K].data_ptr(), self.f_true.data_ptr(), 1.0 / cnt, self.gf.data_ptr(),
                  self.loss.data_ptr(), s)
        B.tat_fill(self.gq.numel(), 0.0, self.gq.data_ptr(), s)
        for k in range(K - 1, -1, -1):
            # primal block: gf = dL/df_{k+1} -> dL/df_k (residual + input 0), gAq = dL/d(A* q_{k+1})
            self._net_backward("primal", n, n, 2, self.gf, self.h1p[k], self.h2p[k], self.g_h2p, self.g_h1p,
                               self.f[k], self.Aq[k], None, self.gf, self.gAq, 0b01)
            # (A*)^T = (W_Y / W_X) A: gq += (W_Y/W_X) A gAq
            self._A(self.gAq, self.tmp_y)
            B.tat_axpby_clamp(self.gq.numel(), 1.0, self.gq.data_ptr(), op.W_Y / op.W_X, self.tmp_y.data_ptr(),
                              -math.inf, 0, 1, self.gq.data_ptr(), s)
            # dual block: gq = dL/dq_{k+1} -> dL/dq_k, gAf = dL/d(A f_k)
            self._net_backward("dual", nd, nt, 3, self.gq, self.h1d[k], self.h2d[k], self.g_h2d, self.g_h1d,
                               self.q[k], self.Af[k], self.y, self.gq, self.gAf, 0b01)
            # A^T = (W_X / W_Y) A*: gf += (W_X/W_Y) A* gAf
            self._Astar(self.gAf, self.tmp_x)
            B.tat_axpby_clamp(self.gf.numel(), 1.0, self.gf.data_ptr(), op.W_X / op.W_Y, self.tmp_x.data_ptr(),
                              -math.inf, 0, 1, self.gf.data_ptr(), s)

    def _adam(self):
        self.t += 1
        B.tat_adam(NPARAM, self.lr, self.betas[0], self.betas[1], self.eps, self.t, self.params.data_ptr(),
                   self.grad.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.wbf.data_ptr(), self._s())

    def loss_and_grad(self, y, f_true):
        """Forward, loss (Eq. emp_loss, mean over pixels and batch) and parameter gradient."""
        self.y.copy_(y)
        self.f_true.copy_(f_true)
        self._forward()
        self._backward()
        return self.loss, self.grad

    def train_step(self, y, f_true, graph=False):
        """One Adam step on the batch (y, f_true); returns the device loss tensor (before the step).

        With graph=True the forward and backward kernels (about 2K operator
        applications of each kind and 12K convolution launches) are captured
        once as a CUDA graph and replayed; the Adam step runs after the replay,
        outside the graph, because its bias correction depends on the step count."""
        self.y.copy_(y)
        self.f_true.copy_(f_true)
        if graph:
            if self._graph is None:
                self._forward()
                self._backward()
                torch.cuda.current_stream(self.dev).synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g):
                    self._forward()
                    self._backward()
                self._graph = g
            self._graph.replay()
        else:
            self._forward()
            self._backward()
        self._adam()
        return self.loss

    def fit(self, f_train, y_train, steps, seed=0, graph=True, log_every=100):
        """Adam on random batches (with replacement, seeded) of the training pairs
        (f_train (N, n, n), y_train (N, n_det, n_t), device tensors); returns
        [(step, loss)] every `log_every` steps and at the last one.  At those points it
        also reads the convolutions' timeout flag and raises TatError if one was set."""
        gen = torch.Generator().manual_seed(seed)
        curve = []
        for it in range(steps):
            idx = torch.randint(0, f_train.shape[0], (self.B,), generator=gen).to(self.dev)
            loss = self.train_step(y_train[idx].contiguous(), f_train[idx].contiguous(), graph=graph)
            if it % log_every == 0 or it == steps - 1:
                curve.append((it, float(loss.item())))
                B.tat_lpd_check()  # raises if a convolution gave up waiting for a tile (no results from it)
        return curve
