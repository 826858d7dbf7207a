"""FP64 CPU oracle of the learned primal-dual reconstruction (Section 4.2.1,
Eqs. LPD_dual, LPD_primal, emp_loss).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path and imports nothing from it.

Plain PyTorch CPU ops in float64; the 3x3 convolutions are
``torch.nn.functional.conv2d`` (a library primitive; cross-correlation with
zero padding), A and A* are the FP64 oracle's (``oracle.solvers.plan_op``), and
the gradients come from autograd.

    q_{k+1} = q_k + Gamma(q_k, A f_k, y),   f_{k+1} = f_k + Lambda(f_k, A* q_{k+1}),
    f_0 = q_0 = 0, k = 0..K-1, weights shared by the iterations; loss = mean (f_K - f)^2.
    Gamma, Lambda: conv3x3(cin -> 32) + ReLU, conv3x3(32 -> 32) + ReLU, conv3x3(32 -> 1),
    added to the residual (q or f).

Readings: the residual form and the zero initial state follow the learned
primal-dual method the paper cites (Adler and Oektem); the nets' size is the
3-layer 32-channel stand-in for the paper's U-Nets (the paper's 3.9 M-parameter
U-Nets need its 10 000-image training set and ~25 h).

With ``bf16=True`` the oracle rounds to BF16 (round to nearest even) exactly
where the CUDA path stores BF16: the inputs of every convolution, the weights,
the two hidden activations and the gradients of the hidden activations; the
rest stays in float64.  With ``bf16=False`` it is the plain float64 network.

The parameter vector is the flat layout of the CUDA path: per net (dual with
cin = 3, then primal with cin = 2) w_in [9][cin][32], b_in [32], w_mid
[9][32 out][32 in], b_mid [32], w_out [9][32], b_out [1], each entry starting
at a multiple of 8 elements.
"""
from __future__ import annotations

import torch
import torch.nn.functional as F

C = 32


def layout():
    """{(net, name): (offset, count)} and the total length of the flat parameter vector."""
    off, table = 0, {}
    for net, cin in (("dual", 3), ("primal", 2)):
        for name, cnt in (("w_in", 9 * cin * C), ("b_in", C), ("w_mid", 9 * C * C), ("b_mid", C),
                          ("w_out", 9 * C), ("b_out", 1)):
            table[(net, name)] = (off, cnt)
            off += (cnt + 7) // 8 * 8
    return table, off


def _round_bf16(x):
    return x.to(torch.bfloat16).to(torch.float64)


class _RoundBoth(torch.autograd.Function):
    """BF16 rounding of a stored tensor and of the gradient that flows back into it."""

    @staticmethod
    def forward(ctx, x):
        return _round_bf16(x)

    @staticmethod
    def backward(ctx, g):
        return _round_bf16(g)


class _RoundForward(torch.autograd.Function):
    """BF16 rounding of an operand as it is read (the gradient passes unchanged)."""

    @staticmethod
    def forward(ctx, x):
        return _round_bf16(x)

    @staticmethod
    def backward(ctx, g):
        return g


def _weights(p, table, net, cin, bf16):
    """torch conv2d weights (out, in, 3, 3) from the flat layouts."""
    def get(name):
        off, cnt = table[(net, name)]
        return p[off:off + cnt]

    rw = _RoundForward.apply if bf16 else (lambda t: t)
    w_in = rw(get("w_in")).reshape(3, 3, cin, C).permute(3, 2, 0, 1)      # [tap][ci][co] -> (co, ci, ky, kx)
    w_mid = rw(get("w_mid")).reshape(3, 3, C, C).permute(2, 3, 0, 1)      # [tap][co][ci] -> (co, ci, ky, kx)
    w_out = rw(get("w_out")).reshape(3, 3, C).permute(2, 0, 1).unsqueeze(0)  # [tap][ci] -> (1, ci, ky, kx)
    return w_in, get("b_in"), w_mid, get("b_mid"), w_out, get("b_out")


def net(p, table, name, cin, planes, residual, bf16=True):
    """One block: residual + conv_out(relu(conv_mid(relu(conv_in(planes))))) on (B, H, W) planes."""
    w_in, b_in, w_mid, b_mid, w_out, b_out = _weights(p, table, name, cin, bf16)
    x = torch.stack(planes, dim=1)
    if bf16:
        x = _RoundForward.apply(x)
    h1 = F.relu(F.conv2d(x, w_in, b_in, padding=1))
    if bf16:
        h1 = _RoundBoth.apply(h1)
    h2 = F.relu(F.conv2d(h1, w_mid, b_mid, padding=1))
    if bf16:
        h2 = _RoundBoth.apply(h2)
    return residual + F.conv2d(h2, w_out, b_out, padding=1)[:, 0]


def reconstruct(p, op, y, K, bf16=True):
    """f_K of K learned primal-dual iterations (Eqs. LPD_dual, LPD_primal) for data y (B, n_det, n_t)."""
    table, _ = layout()
    n = op.x_shape[-1]
    f = torch.zeros((y.shape[0], n, n), dtype=torch.float64)
    q = torch.zeros_like(y)
    for _ in range(K):
        q = net(p, table, "dual", 3, [q, op.A(f), y], q, bf16)
        f = net(p, table, "primal", 2, [f, op.Astar(q)], f, bf16)
    return f


def loss(p, op, y, f_true, K, bf16=True):
    """Eq. emp_loss for one batch: mean over images and pixels of (f_K - f)^2."""
    f = reconstruct(p, op, y, K, bf16)
    return ((f - f_true) ** 2).mean()


def loss_and_grad(p, op, y, f_true, K, bf16=True):
    """(loss, d loss / d p) by autograd of the float64 network."""
    p = p.detach().clone().requires_grad_(True)
    L = loss(p, op, y, f_true, K, bf16)
    (g,) = torch.autograd.grad(L, p)
    return float(L.detach()), g
