"""Pins of the FP64 oracle of the learned primal-dual reconstruction (Section 4.2.1).

The network is pinned against computations that do not go through it: with
hand-set weights the blocks reduce to known linear maps (a one-pixel shift of
the data, and a linear primal-dual iteration written out with the oracle's A
and A*), which fixes the tap orientation, the channel order, the residual form
and the order of the updates in Eqs. LPD_dual and LPD_primal; finite
differences check the autograd gradient of Eq. emp_loss; and the BF16
emulation changes the loss by a BF16-sized amount only.
"""
import math

import numpy as np
import torch

from oracle import lpd as L
from oracle import solvers as S
from oracle import tat_oracle as O
from tat_inputs import ellipse_phantom, gaussian

F64 = torch.float64


def _op(n=12, nd=16, nt=16):
    P = O.OraclePlan(n, nd, nt, support_radius=0.9)
    return P, S.plan_op(P)


def _set(p, table, net, name, idx, value):
    off, cnt = table[(net, name)]
    assert 0 <= idx < cnt
    p[off + idx] = value


def _passthrough(p, table, net, cin, coef, tap_in=4):
    """Block output = sum_c coef[c] * x_c at tap `tap_in` (ReLU pairs h = relu(s), relu(-s))."""
    for c, a in enumerate(coef):
        _set(p, table, net, "w_in", (tap_in * cin + c) * 32 + 0, a)
        _set(p, table, net, "w_in", (tap_in * cin + c) * 32 + 1, -a)
    for ch in (0, 1):
        _set(p, table, net, "w_mid", (4 * 32 + ch) * 32 + ch, 1.0)     # centre tap, identity on channels 0, 1
    _set(p, table, net, "w_out", 4 * 32 + 0, 1.0)
    _set(p, table, net, "w_out", 4 * 32 + 1, -1.0)


def test_tap_orientation_and_channels():
    """Dual block = y shifted by one detector (tap dy = +1), primal block = A* q: f_1 = A*(y(d+1, m))."""
    P, op = _op()
    table, npar = L.layout()
    p = torch.zeros(npar, dtype=F64)
    _passthrough(p, table, "dual", 3, [0.0, 0.0, 1.0], tap_in=7)        # tap 7: dy = +1, dx = 0
    _passthrough(p, table, "primal", 2, [0.0, 1.0])
    y = torch.tensor(gaussian(3, 2 * 16 * 16).reshape(2, 16, 16))
    f1 = L.reconstruct(p, op, y, K=1, bf16=False)
    ys = torch.zeros_like(y)
    ys[:, :-1, :] = y[:, 1:, :]
    ref = op.Astar(ys)
    assert float((f1 - ref).abs().max()) <= 1e-12 * float(ref.abs().max())


def test_linear_primal_dual_iteration():
    """With linear blocks the network is the iteration q <- q + a q + b A f + c y, f <- f + d f + e A* q_new."""
    P, op = _op()
    table, npar = L.layout()
    p = torch.zeros(npar, dtype=F64)
    a, b, c, d, e = -0.3, 0.7, -0.7, -0.1, -0.4
    _passthrough(p, table, "dual", 3, [a, b, c])
    _passthrough(p, table, "primal", 2, [d, e])
    f_true = torch.tensor(np.stack([ellipse_phantom(12, s) for s in (1, 2)]))
    y = op.A(f_true)
    fK = L.reconstruct(p, op, y, K=3, bf16=False)
    f = torch.zeros_like(f_true)
    q = torch.zeros_like(y)
    for _ in range(3):
        q = q + a * q + b * op.A(f) + c * y
        f = f + d * f + e * op.Astar(q)
    assert float((fK - f).abs().max()) <= 1e-12 * float(f.abs().max())


def test_loss_gradient_finite_differences():
    """d(Eq. emp_loss)/d(parameters) by central differences along a random direction (float64, no BF16)."""
    P, op = _op(8, 12, 12)
    table, npar = L.layout()
    p = torch.tensor(0.1 * gaussian(11, npar))
    f_true = torch.tensor(np.stack([ellipse_phantom(8, s) for s in (4, 5)]))
    y = op.A(f_true)
    _, g = L.loss_and_grad(p, op, y, f_true, K=2, bf16=False)
    v = torch.tensor(gaussian(12, npar))
    eps = 1e-6
    fd = (L.loss(p + eps * v, op, y, f_true, 2, False) - L.loss(p - eps * v, op, y, f_true, 2, False)) / (2 * eps)
    ad = float((g * v).sum())
    assert abs(ad - float(fd)) <= 1e-6 * abs(float(fd))


def test_bf16_emulation_is_bf16_sized():
    """Rounding at the BF16 storage points moves the loss by a relative amount of BF16 size."""
    P, op = _op(8, 12, 12)
    table, npar = L.layout()
    p = torch.tensor(0.1 * gaussian(21, npar))
    f_true = torch.tensor(np.stack([ellipse_phantom(8, s) for s in (6, 7)]))
    y = op.A(f_true)
    l64 = float(L.loss(p, op, y, f_true, 2, bf16=False))
    l16 = float(L.loss(p, op, y, f_true, 2, bf16=True))
    assert 1e-6 < abs(l16 - l64) / l64 < 5e-2
    assert math.isfinite(l16)
