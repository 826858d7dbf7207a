"""Pins of the FP64 solver oracle (Section 4.2) against what the mathematics fixes.

Each check uses something other than the oracle itself: a brute-force matrix
of the difference operators, the closed-form spectrum of the discrete
gradient, SciPy's active-set NNLS, the closed-form 1-D total-variation
denoising of a step, and central finite differences of the unrolled
iterations in float64.
"""
import math

import numpy as np
import pytest
import torch
from scipy.optimize import nnls as scipy_nnls

from oracle import solvers as S
from oracle import tat_oracle as O
from tat_inputs import ellipse_phantom, gaussian, roi_mask, uniform

F64 = torch.float64


def _t(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float64))


def _grad_matrix(n, h):
    cols = [S.grad_h(_t(np.eye(n * n)[i].reshape(n, n)), h).reshape(-1) for i in range(n * n)]
    return torch.stack(cols, dim=1).numpy()


def _div_matrix(n, h):
    cols = [S.div_h(_t(np.eye(2 * n * n)[i].reshape(2, n, n)), h).reshape(-1) for i in range(2 * n * n)]
    return torch.stack(cols, dim=1).numpy()


# ------------------------------------------------------------ difference operators

def test_grad_of_ramps():
    """grad_h of f = x is (1, 0) except the zero last column; of f = y, (0, 1) except the last row."""
    n = 7
    h = 2.0 / (n - 1)
    x = -1 + h * np.arange(n)
    gx = S.grad_h(_t(np.tile(x, (n, 1))), h).numpy()
    assert np.allclose(gx[0, :, :-1], 1.0) and np.allclose(gx[0, :, -1], 0.0) and np.allclose(gx[1], 0.0)
    gy = S.grad_h(_t(np.tile(x[:, None], (1, n))), h).numpy()
    assert np.allclose(gy[1, :-1, :], 1.0) and np.allclose(gy[1, -1, :], 0.0) and np.allclose(gy[0], 0.0)


def test_div_is_minus_grad_transpose():
    """Brute force: the matrix of div_h equals minus the transpose of the matrix of grad_h."""
    n, h = 5, 0.37
    G, D = _grad_matrix(n, h), _div_matrix(n, h)
    assert np.abs(D + G.T).max() < 1e-13


def test_grad_norm_closed_form():
    """||grad_h||^2 = 8 sin^2(pi (n-1) / (2n)) / h^2 (eigenvalues of the Neumann difference Laplacian),
    reached by the oracle's power iteration."""
    n, h = 6, 0.25
    op = S.LinearOp(lambda f: S.grad_h(_t(f), h).numpy(), lambda p: (-S.div_h(_t(p), h)).numpy(),
                    (n, n), (2, n, n))
    v0 = _t(uniform(3, n * n).reshape(n, n) - 0.5)
    est = S.power_norm_sq(op, v0, 400)
    exact = 8.0 * math.sin(math.pi * (n - 1) / (2 * n)) ** 2 / h ** 2
    assert abs(est - exact) / exact < 1e-10
    assert np.linalg.norm(_grad_matrix(n, h), 2) ** 2 == pytest.approx(exact, rel=1e-12)


# ------------------------------------------------------------ NNLS

def _dense_problem(seed, m=40, n=5):
    M = gaussian(seed, m * n * n).reshape(m, n * n)
    f_true = uniform(seed + 1, n * n) - 0.3
    g = M @ f_true + 0.1 * gaussian(seed + 2, m)
    return M, g


def test_nnls_matches_scipy():
    """Projected gradient with lambda = 1/||A||^2 converges to SciPy's active-set NNLS solution."""
    n = 5
    M, g = _dense_problem(11)
    op = S.matrix_op(M, n)
    L = np.linalg.norm(M, 2) ** 2
    assert S.power_norm_sq(op, _t(uniform(5, n * n).reshape(n, n)), 500) == pytest.approx(L, rel=1e-9)
    f = S.nnls(op, _t(g), 1.0 / L, 4000).numpy().reshape(-1)
    ref, _ = scipy_nnls(M, g)
    assert (ref == 0).sum() >= 3, "the test problem should have active constraints"
    assert np.abs(f - ref).max() < 1e-9


def test_nnls_mask_is_restriction():
    """With Pi_Omega0 the iteration solves NNLS over the masked pixels only (zero elsewhere)."""
    n = 5
    M, g = _dense_problem(21)
    mask = roi_mask(n, radius=0.9, upper_half=True)
    keep = mask.reshape(-1) > 0
    op = S.matrix_op(M, n)
    L = np.linalg.norm(M, 2) ** 2
    f = S.nnls(op, _t(g), 1.0 / L, 4000, mask=_t(mask)).numpy().reshape(-1)
    ref = np.zeros(n * n)
    ref[keep], _ = scipy_nnls(M[:, keep], g)
    assert np.abs(f - ref).max() < 1e-9
    assert np.all(f[~keep] == 0)


def test_roi_mask_half_disk():
    """The upper half disk: y >= 0 and |x| <= radius on the node grid."""
    m = roi_mask(9, radius=1.0, upper_half=True)
    assert m[:4].sum() == 0 and m[4].sum() == 9 and m[8, 4] == 1 and m[8, 0] == 0


# ------------------------------------------------------------ TV-PDHG

def test_pdhg_tv_denoise_step_closed_form():
    """A = I, g a step in x constant in y: each row solves 1-D TV denoising, whose solution moves the
    two levels towards each other by beta/m and beta/(n-m), beta = alpha/h."""
    n, m, h, alpha = 8, 3, 0.5, 0.05
    a, b = 1.0, 2.0
    g = np.where(np.arange(n) < m, a, b)[None, :].repeat(n, 0)
    op = S.LinearOp(lambda f: f, lambda y: y, (n, n), (n, n))
    sigma, tau, s = S.pdhg_steps(1.0, h)
    f = S.tv_pdhg(op, _t(g), alpha, h, 6000, sigma, tau, s).numpy()
    beta = alpha / h
    want = np.where(np.arange(n) < m, a + beta / m, b - beta / (n - m))[None, :].repeat(n, 0)
    assert np.abs(f - want).max() < 1e-7


def test_pdhg_positivity_and_mask():
    """A = I and alpha -> 0: the solution is Pi_Omega0 max(0, g)."""
    n, h = 6, 0.4
    g = gaussian(31, n * n).reshape(n, n)
    mask = roi_mask(n, radius=0.95)
    op = S.LinearOp(lambda f: f, lambda y: y, (n, n), (n, n))
    sigma, tau, s = S.pdhg_steps(1.0, h)
    f = S.tv_pdhg(op, _t(g), 1e-12, h, 3000, sigma, tau, s, mask=_t(mask)).numpy()
    assert np.abs(f - np.maximum(g, 0) * mask).max() < 1e-8


def test_pdhg_without_tv_is_nnls():
    """alpha -> 0 with a dense A: PDHG reaches SciPy's NNLS solution."""
    n = 5
    M, g = _dense_problem(41)
    op = S.matrix_op(M, n)
    L = np.linalg.norm(M, 2) ** 2
    sigma, tau, s = S.pdhg_steps(L, 0.5)
    f = S.tv_pdhg(op, _t(g), 1e-12, 0.5, 20000, sigma, tau, s).numpy().reshape(-1)
    ref, _ = scipy_nnls(M, g)
    assert np.abs(f - ref).max() < 1e-6


def test_pdhg_decreases_tv_objective():
    """On a small oracle operator PDHG drives the TV objective below its value at the true image
    (a feasible point, so an upper bound of the minimum) and keeps lowering it."""
    P = O.OraclePlan(16, 32, 32)
    op = S.plan_op(P)
    f_true = _t(ellipse_phantom(16, 3))
    g = op.A(f_true)
    L = S.power_norm_sq(op, _t(uniform(7, 256).reshape(16, 16)), 30)
    sigma, tau, s = S.pdhg_steps(L * 1.05, P.h)
    alpha = 1e-3
    obj = [float(S.tv_objective(op, S.tv_pdhg(op, g, alpha, P.h, it, sigma, tau, s), g, alpha, P.h, P.W_Y, P.W_X))
           for it in (30, 60)]
    obj_true = float(S.tv_objective(op, f_true, g, alpha, P.h, P.W_Y, P.W_X))
    assert obj[1] < obj[0] < obj_true


# ------------------------------------------------------------ differentiation

def _fd_check(fun, x, seed, eps=1e-6, tol=1e-6):
    x = x.clone().requires_grad_(True)
    y = fun(x)
    w = _t(gaussian(seed, y.numel()).reshape(y.shape))
    (gx,) = torch.autograd.grad((w * y).sum(), x)
    v = _t(gaussian(seed + 1, x.numel()).reshape(x.shape))
    with torch.no_grad():
        fd = ((w * fun(x + eps * v)).sum() - (w * fun(x - eps * v)).sum()) / (2 * eps)
    ad = (gx * v).sum()
    assert abs(float(ad) - float(fd)) <= tol * max(1.0, abs(float(fd))), (float(ad), float(fd))


def test_operator_transpose_weights_fd():
    """d<w, A f>/df and d<w, A* g>/dg by finite differences: pins A^T = (W_X/W_Y) A* in the backward."""
    P = O.OraclePlan(12, 16, 16, arc_len=math.pi)
    op = S.plan_op(P)
    _fd_check(op.A, _t(ellipse_phantom(12, 1)), 51, eps=1e-3, tol=1e-9)
    _fd_check(op.Astar, _t(gaussian(60, 16 * 16).reshape(16, 16)), 53, eps=1e-3, tol=1e-9)


def test_unrolled_nnls_gradient_fd():
    """Gradient of an unrolled NNLS solve with respect to the data g, by finite differences."""
    n = 5
    M, g = _dense_problem(71)
    op = S.matrix_op(M, n)
    lam = 1.0 / np.linalg.norm(M, 2) ** 2
    mask = _t(roi_mask(n, radius=0.95))
    _fd_check(lambda gg: S.nnls(op, gg, lam, 12, mask=mask), _t(g), 81)


def test_unrolled_pdhg_gradient_fd():
    """Gradient of unrolled TV-PDHG with respect to g, by finite differences."""
    n = 5
    M, g = _dense_problem(91)
    op = S.matrix_op(M, n)
    L = np.linalg.norm(M, 2) ** 2
    sigma, tau, s = S.pdhg_steps(L, 0.5)
    _fd_check(lambda gg: S.tv_pdhg(op, gg, 0.05, 0.5, 12, sigma, tau, s), _t(g), 101)
