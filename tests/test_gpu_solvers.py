"""GPU parity of the solver steps, the autograd Functions and the NNLS / TV-PDHG
iterations (Section 4.2) against the FP64 oracle of ``oracle/solvers.py``.

Bars: element-wise steps and their backward passes <= 1e-6 relative L2 (one
FP32 rounding per operation); anything that applies A or A* <= 1e-5 relative
L2 per application, and a few iterations stay within 1e-5 because each step
is non-expansive; gradients through unrolled iterations <= 1e-4.
"""
import math

import numpy as np
import pytest

from oracle import solvers as S
from oracle import tat_oracle as O
from tat_inputs import add_noise, ellipse_phantom, gaussian, roi_mask, uniform

pytestmark = pytest.mark.gpu

CFG = dict(n=64, n_det=128, n_t=128, support_radius=0.9, arc_begin=0.0, arc_len=math.pi)


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_24687_gb300 as p
    return p


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return t


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def dev(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda:0")


def t64(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float64))


@pytest.fixture(scope="module")
def setup(pkg, torch):
    kw = dict(CFG)
    n, nd, nt = kw.pop("n"), kw.pop("n_det"), kw.pop("n_t")
    op = pkg.TatOperator(n, nd, nt, device="cuda:0", **kw)
    P = O.OraclePlan(n, nd, nt, **kw)
    oop = S.plan_op(P)
    mask = roi_mask(n, radius=0.9, upper_half=True)
    f_true = f32(ellipse_phantom(n, 5))
    g = f32(add_noise(O.forward(P, f_true), 0.01, 6))
    L = pkg.power_norm_sq(op, iters=40)
    return dict(op=op, P=P, oop=oop, mask=mask, g=g, L=L, n=n)


# ------------------------------------------------------------ element-wise steps

def test_power_norm_sq_is_close_to_oracle(pkg, torch, setup):
    """The GPU power iteration and the oracle's agree on ||A||^2 (different start vectors)."""
    n = setup["n"]
    ref = S.power_norm_sq(setup["oop"], t64(torch, uniform(1, n * n).reshape(n, n) - 0.5), 40)
    assert abs(setup["L"] - ref) / ref < 5e-2


def test_axpby_clamp_and_backward(pkg, torch):
    n, B = 37, 3
    x, y = f32(gaussian(1, B * n * n)), f32(gaussian(2, B * n * n))
    mask = roi_mask(n, 0.8, upper_half=True)
    a, b = 0.75, -1.25
    xt, yt = dev(torch, x).reshape(B, n, n), dev(torch, y).reshape(B, n, n)
    xt.requires_grad_(True)
    yt.requires_grad_(True)
    out = pkg.autograd.AxpbyClampFn.apply(xt, yt, a, b, 0.0, dev(torch, mask))
    X, Y = t64(torch, x).reshape(B, n, n).requires_grad_(True), t64(torch, y).reshape(B, n, n).requires_grad_(True)
    ref = torch.clamp(a * X + b * Y, min=0.0) * t64(torch, mask)
    assert rel(out.detach().cpu().numpy(), ref.detach().numpy()) <= 1e-6
    w = f32(gaussian(3, B * n * n)).reshape(B, n, n)
    gx, gy = torch.autograd.grad((out * dev(torch, w)).sum(), (xt, yt))
    rx, ry = torch.autograd.grad((ref * t64(torch, w)).sum(), (X, Y))
    assert rel(gx.cpu().numpy(), rx.numpy()) <= 1e-6 and rel(gy.cpu().numpy(), ry.numpy()) <= 1e-6


def test_pd_dual_data_and_backward(pkg, torch):
    m, sigma = 4097, 0.37
    q, Af, g = (f32(gaussian(s, m)) for s in (11, 12, 13))
    ins = [dev(torch, v).requires_grad_(True) for v in (q, Af, g)]
    refs = [t64(torch, v).requires_grad_(True) for v in (q, Af, g)]
    out = pkg.autograd.PdDualDataFn.apply(*ins, sigma)
    ref = S.pdhg_dual_data(*refs, sigma)
    assert rel(out.detach().cpu().numpy(), ref.detach().numpy()) <= 1e-6
    w = f32(gaussian(14, m))
    gd = torch.autograd.grad((out * dev(torch, w)).sum(), ins)
    gr = torch.autograd.grad((ref * t64(torch, w)).sum(), refs)
    for a, b in zip(gd, gr):
        assert rel(a.cpu().numpy(), b.numpy()) <= 1e-6


@pytest.mark.parametrize("n,B", [(5, 1), (64, 2), (131, 3)])
def test_tv_dual_and_backward(pkg, torch, n, B):
    h, sigma, alpha, s = 2.0 / (n - 1), 0.4, 0.05, 0.7
    p = f32(0.03 * gaussian(21, B * 2 * n * n)).reshape(B, 2, n, n)
    fb = f32(0.2 * h * uniform(22, B * n * n)).reshape(B, n, n)
    pt, ft = dev(torch, p).requires_grad_(True), dev(torch, fb).requires_grad_(True)
    out = pkg.autograd.TvDualFn.apply(pt, ft, sigma, alpha / s, h / s)
    P64, F64 = t64(torch, p).requires_grad_(True), t64(torch, fb).requires_grad_(True)
    ref = S.tv_dual(P64, F64, sigma, alpha, s, h)
    frac = float((torch.linalg.vector_norm(ref.detach(), dim=1) >= alpha / s * (1 - 1e-9)).double().mean())
    assert 0.05 < frac < 0.95, "the projection should be active on part of the image"
    assert rel(out.detach().cpu().numpy(), ref.detach().numpy()) <= 1e-6
    w = f32(gaussian(23, B * 2 * n * n)).reshape(B, 2, n, n)
    gp, gf = torch.autograd.grad((out * dev(torch, w)).sum(), (pt, ft))
    rp, rf = torch.autograd.grad((ref * t64(torch, w)).sum(), (P64, F64))
    assert rel(gp.cpu().numpy(), rp.numpy()) <= 1e-6
    assert rel(gf.cpu().numpy(), rf.numpy()) <= 1e-6


@pytest.mark.parametrize("n,B,masked", [(5, 1, False), (64, 2, True), (131, 3, True)])
def test_tv_primal_and_backward(pkg, torch, n, B, masked):
    h, tau, s = 2.0 / (n - 1), 0.3, 0.7
    f = f32(uniform(31, B * n * n)).reshape(B, n, n)
    Asq = f32(gaussian(32, B * n * n)).reshape(B, n, n)
    p = f32(0.2 * gaussian(33, B * 2 * n * n)).reshape(B, 2, n, n)
    mask = roi_mask(n, 0.9, upper_half=True) if masked else None
    ins = [dev(torch, v).requires_grad_(True) for v in (f, Asq, p)]
    refs = [t64(torch, v).requires_grad_(True) for v in (f, Asq, p)]
    fn, fb = pkg.autograd.TvPrimalFn.apply(*ins, tau, h / s, dev(torch, mask) if masked else None)
    rn, rb = S.tv_primal(*refs, tau, s, h, t64(torch, mask) if masked else None)
    assert rel(fn.detach().cpu().numpy(), rn.detach().numpy()) <= 1e-6
    assert rel(fb.detach().cpu().numpy(), rb.detach().numpy()) <= 1e-6
    w1, w2 = (f32(gaussian(sd, B * n * n)).reshape(B, n, n) for sd in (34, 35))
    gd = torch.autograd.grad((fn * dev(torch, w1)).sum() + (fb * dev(torch, w2)).sum(), ins)
    gr = torch.autograd.grad((rn * t64(torch, w1)).sum() + (rb * t64(torch, w2)).sum(), refs)
    for a, b in zip(gd, gr):
        assert rel(a.cpu().numpy(), b.numpy()) <= 1e-6


# ------------------------------------------------------------ operator autograd

def test_operator_autograd_vs_oracle(pkg, torch, setup):
    """Backward of A is (W_X/W_Y) A*, backward of A* is (W_Y/W_X) A: compared with the oracle's autograd."""
    op, oop, n = setup["op"], setup["oop"], setup["n"]
    f = f32(ellipse_phantom(n, 7))
    w = f32(gaussian(8, op.n_det * op.n_t)).reshape(op.n_det, op.n_t)
    ft = dev(torch, f).requires_grad_(True)
    (gd,) = torch.autograd.grad((pkg.A(op, ft) * dev(torch, w)).sum(), ft)
    F = t64(torch, f).requires_grad_(True)
    (gr,) = torch.autograd.grad((oop.A(F) * t64(torch, w)).sum(), F)
    assert rel(gd.cpu().numpy(), gr.numpy()) <= 1e-5
    v = f32(gaussian(9, n * n)).reshape(n, n)
    gt = dev(torch, w).requires_grad_(True)
    (hd,) = torch.autograd.grad((pkg.Astar(op, gt) * dev(torch, v)).sum(), gt)
    G = t64(torch, w).requires_grad_(True)
    (hr,) = torch.autograd.grad((oop.Astar(G) * t64(torch, v)).sum(), G)
    assert rel(hd.cpu().numpy(), hr.numpy()) <= 1e-5


# ------------------------------------------------------------ iterations

def test_nnls_iterations_vs_oracle(pkg, torch, setup):
    op, oop, mask, g, L = setup["op"], setup["oop"], setup["mask"], setup["g"], setup["L"]
    lam = 1.0 / L
    solver = pkg.TatSolver(op, 1, mask=dev(torch, mask))
    fd = solver.nnls(dev(torch, g)[None], 8, lam).cpu().numpy()[0]
    fr = S.nnls(oop, t64(torch, g), lam, 8, mask=t64(torch, mask)).numpy()
    assert rel(fd, fr) <= 1e-5
    assert fd.min() >= 0 and np.all(fd[mask == 0] == 0)
    fgraph = solver.nnls(dev(torch, g)[None], 8, lam, graph=True).cpu().numpy()[0]
    assert rel(fgraph, fd) <= 1e-6


def test_tv_iterations_vs_oracle(pkg, torch, setup):
    op, oop, mask, g, L, P = setup["op"], setup["oop"], setup["mask"], setup["g"], setup["L"], setup["P"]
    sigma, tau, s = pkg.pdhg_steps(L * 1.05, P.h)
    alpha = 1e-3
    solver = pkg.TatSolver(op, 1, mask=dev(torch, mask), h=P.h)
    fd = solver.tv(dev(torch, g)[None], alpha, 8, sigma, tau, s).cpu().numpy()[0]
    fr = S.tv_pdhg(oop, t64(torch, g), alpha, P.h, 8, sigma, tau, s, mask=t64(torch, mask)).numpy()
    assert rel(fd, fr) <= 1e-5
    fgraph = solver.tv(dev(torch, g)[None], alpha, 8, sigma, tau, s, graph=True).cpu().numpy()[0]
    assert rel(fgraph, fd) <= 1e-6


def test_batched_solver_matches_single(pkg, torch, setup):
    op, P, L, mask = setup["op"], setup["P"], setup["L"], setup["mask"]
    gs = np.stack([f32(add_noise(O.forward(P, ellipse_phantom(P.n, 40 + b)), 0.01, 50 + b)) for b in range(3)])
    batched = pkg.TatSolver(op, 3, mask=dev(torch, mask)).nnls(dev(torch, gs), 5, 1.0 / L).cpu().numpy()
    single = pkg.TatSolver(op, 1, mask=dev(torch, mask))
    for b in range(3):
        fb = single.nnls(dev(torch, gs[b])[None], 5, 1.0 / L).cpu().numpy()[0]
        assert rel(batched[b], fb) <= 1e-6


def test_unrolled_nnls_gradient_vs_oracle(pkg, torch, setup):
    op, oop, mask, g, L = setup["op"], setup["oop"], setup["mask"], setup["g"], setup["L"]
    lam, it = 1.0 / L, 3
    n = setup["n"]
    w = f32(gaussian(61, n * n)).reshape(n, n)
    gt = dev(torch, g).requires_grad_(True)
    fd = pkg.nnls_unrolled(op, gt, it, lam, mask=dev(torch, mask))
    (gd,) = torch.autograd.grad((fd * dev(torch, w)).sum(), gt)
    G = t64(torch, g).requires_grad_(True)
    fr = S.nnls(oop, G, lam, it, mask=t64(torch, mask))
    (gr,) = torch.autograd.grad((fr * t64(torch, w)).sum(), G)
    assert rel(fd.detach().cpu().numpy(), fr.detach().numpy()) <= 1e-5
    assert rel(gd.cpu().numpy(), gr.numpy()) <= 1e-4


def test_unrolled_tv_gradient_vs_oracle(pkg, torch, setup):
    op, oop, mask, g, L, P = setup["op"], setup["oop"], setup["mask"], setup["g"], setup["L"], setup["P"]
    sigma, tau, s = pkg.pdhg_steps(L * 1.05, P.h)
    alpha, it = 1e-3, 3
    n = setup["n"]
    w = f32(gaussian(71, n * n)).reshape(n, n)
    gt = dev(torch, g).requires_grad_(True)
    fd = pkg.tv_unrolled(op, gt, alpha, it, sigma, tau, s, mask=dev(torch, mask), h=P.h)
    (gd,) = torch.autograd.grad((fd * dev(torch, w)).sum(), gt)
    G = t64(torch, g).requires_grad_(True)
    fr = S.tv_pdhg(oop, G, alpha, P.h, it, sigma, tau, s, mask=t64(torch, mask))
    (gr,) = torch.autograd.grad((fr * t64(torch, w)).sum(), G)
    assert rel(fd.detach().cpu().numpy(), fr.detach().numpy()) <= 1e-5
    assert rel(gd.cpu().numpy(), gr.numpy()) <= 1e-4


def test_invalid_solver_arguments(pkg, torch, setup):
    with pytest.raises(pkg.TatError):
        pkg.tat_tv_dual(1, 8, 0.0, 1.0, 1.0, 1, 1, 1)     # h_eff = 0
    with pytest.raises(pkg.TatError):
        pkg.tat_pd_dual_data(0, 1.0, 1, 1, 1, 1)          # empty
    with pytest.raises(ValueError):
        pkg.TatSolver(setup["op"], 1).nnls(torch.zeros((2, 128, 128), device="cuda:0"), 1, 1.0)


# ------------------------------------------------------------ solves workload (full size)

def test_solves_workload_full_size(pkg, torch):
    """B = 16, n = 256, 512 detectors on a half circle, n_t = 512, 1 % noise.

    Parity: two NNLS iterations and two PDHG iterations of batch entry 0 against the oracle.
    Properties of the 100-iteration solves: f >= 0, zero outside Omega_0, monotone NNLS residual,
    decreasing TV objective."""
    n, nd, nt, B = 256, 512, 512, 16
    kw = dict(support_radius=0.9, arc_begin=0.0, arc_len=math.pi)
    op = pkg.TatOperator(n, nd, nt, device="cuda:0", **kw)
    P = O.OraclePlan(n, nd, nt, **kw)
    oop = S.plan_op(P)
    mask = roi_mask(n, radius=0.9, upper_half=True)
    f_true = np.stack([f32(ellipse_phantom(n, b)) for b in range(B)])
    g0 = f32(add_noise(O.forward(P, f_true[0]), 0.01, 1000))
    gd = op.forward(dev(torch, f_true)).cpu().numpy()
    g = np.stack([g0] + [f32(add_noise(gd[b], 0.01, 1000 + b)) for b in range(1, B)])
    L = pkg.power_norm_sq(op, iters=30)
    solver = pkg.TatSolver(op, B, mask=dev(torch, mask), h=P.h)
    gt = dev(torch, g)

    f2 = solver.nnls(gt, 2, 1.0 / L).cpu().numpy()
    r2 = S.nnls(oop, t64(torch, g0), 1.0 / L, 2, mask=t64(torch, mask)).numpy()
    assert rel(f2[0], r2) <= 1e-5
    sigma, tau, s = pkg.pdhg_steps(L * 1.05, P.h)
    alpha = 1e-3
    t2 = solver.tv(gt, alpha, 2, sigma, tau, s).cpu().numpy()
    rt2 = S.tv_pdhg(oop, t64(torch, g0), alpha, P.h, 2, sigma, tau, s, mask=t64(torch, mask)).numpy()
    assert rel(t2[0], rt2) <= 1e-5

    def resid(f):
        return torch.linalg.vector_norm((op.forward(f) - gt).reshape(B, -1), dim=1)

    prev = resid(torch.zeros((B, n, n), device="cuda:0"))
    for it in (25, 50, 100):
        f = solver.nnls(gt, it, 1.0 / L, graph=True).clone()
        cur = resid(f)
        assert bool((cur <= prev * (1 + 1e-6)).all())
        prev = cur
    fn = f.cpu().numpy()
    assert fn.min() >= 0 and np.all(fn[:, mask == 0] == 0)

    def tv_obj(f):
        r = (op.forward(f) - gt).reshape(B, -1)
        gx = torch.zeros_like(f)
        gy = torch.zeros_like(f)
        gx[:, :, :-1] = (f[:, :, 1:] - f[:, :, :-1]) / P.h
        gy[:, :-1, :] = (f[:, 1:, :] - f[:, :-1, :]) / P.h
        return 0.5 * op.W_Y * (r * r).sum(1) + alpha * op.W_X * torch.sqrt(gx * gx + gy * gy).reshape(B, -1).sum(1)

    o10 = tv_obj(solver.tv(gt, alpha, 10, sigma, tau, s, graph=True).clone())
    o100 = tv_obj(solver.tv(gt, alpha, 100, sigma, tau, s, graph=True).clone())
    assert bool((o100 < o10).all())
    ft = solver.f.cpu().numpy()
    assert ft.min() >= 0 and np.all(ft[:, mask == 0] == 0)
