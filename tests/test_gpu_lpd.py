"""GPU parity of the learned primal-dual kernels (include/tat_lpd.h) and of the
whole unrolled network, forward and backward, against the FP64 oracle with
BF16 rounding at the same storage points (oracle/lpd.py).

Bars (derived from the arithmetic): values stored in BF16 may differ from the
oracle by one BF16 rounding where the FP32 and FP64 accumulations fall on
opposite sides of a rounding boundary (rare: the accumulations agree to
~1e-6 while a BF16 step is 2^-8 relative), so BF16 outputs are held to 1e-3
relative L2; FP32 outputs computed from identical BF16 operands to 1e-5;
weight gradients (FP32 sums over up to 10^5 products) to 1e-4.  The whole
network, where flips propagate through 3 unrolled iterations, to 2e-3 on the
loss and 2e-2 on the parameter gradient.
"""
import numpy as np
import pytest

from tat_inputs import ellipse_phantom, gaussian, uniform

pytestmark = pytest.mark.gpu


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
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def r16(torch, x):
    return torch.as_tensor(x, dtype=torch.float64).to(torch.bfloat16).to(torch.float64)


def dev_bf16(torch, x):
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).view(torch.int16).cuda().contiguous()


def host_bf16(torch, t):
    return t.view(torch.bfloat16).to(torch.float64).cpu()


def dev32(torch, x):
    return torch.as_tensor(np.asarray(x, np.float32)).cuda().contiguous()


# (2, 20, 36): not multiples of the tiles, one tile per CTA; (2, 200, 264): also ragged, ~850
# tiles against 456-608 persistent CTAs, so CTAs run several tiles through their TMA slots,
# mbarrier phases and TMEM accumulators
LAYER_SIZES = [(2, 20, 36), (2, 200, 264)]
LAYER_IDS = ["ragged", "multi-tile"]


def _stream(torch):
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("cin", [2, 3])
@pytest.mark.parametrize("size", LAYER_SIZES, ids=LAYER_IDS)
def test_conv_in_forward_backward(pkg, torch, cin, size):
    B_, H_, W_ = size
    import torch.nn.functional as F
    xs = [uniform(10 + c, B_ * H_ * W_).reshape(B_, H_, W_) - 0.3 for c in range(cin)]
    w = 0.3 * gaussian(20, 9 * cin * 32)
    b = 0.1 * gaussian(21, 32)
    s = _stream(torch)
    xd = [dev32(torch, x) for x in xs]
    wd, bd = dev_bf16(torch, w), dev32(torch, b)
    h = torch.empty((B_, H_, W_, 32), dtype=torch.int16, device="cuda")
    pkg.tat_conv_in_fwd(B_, H_, W_, cin, xd[0].data_ptr(), xd[1].data_ptr(), xd[2].data_ptr() if cin == 3 else 0,
                        wd.data_ptr(), bd.data_ptr(), h.data_ptr(), s)
    X = r16(torch, np.stack(xs, 1)).requires_grad_(True)
    Wt = r16(torch, w).reshape(3, 3, cin, 32).permute(3, 2, 0, 1).contiguous().requires_grad_(True)
    Bt = torch.tensor(np.asarray(b, np.float32), dtype=torch.float64).requires_grad_(True)
    pre = F.conv2d(X, Wt, Bt, padding=1)
    ref = r16(torch, torch.relu(pre).detach())                                   # (B, 32, H, W)
    assert rel(host_bf16(torch, h).permute(0, 3, 1, 2), ref) <= 1e-3
    # backward: G (BF16) at the output; mask from the device forward
    G = 0.5 * gaussian(30, B_ * H_ * W_ * 32).reshape(B_, H_, W_, 32)
    Gd = dev_bf16(torch, G)
    gx = [torch.full((B_, H_, W_), 7.0, device="cuda") for _ in range(cin)]
    pkg.tat_conv_in_bwd_data(B_, H_, W_, cin, Gd.data_ptr(), h.data_ptr(), wd.data_ptr(), gx[0].data_ptr(),
                             gx[1].data_ptr(), gx[2].data_ptr() if cin == 3 else 0, 0b01, s)
    scratch = torch.empty(pkg.tat_lpd_scratch_floats(B_, H_, W_), device="cuda")
    gw = torch.zeros(9 * cin * 32, device="cuda")
    gb = torch.zeros(32, device="cuda")
    pkg.tat_conv_in_bwd_weights(B_, H_, W_, cin, xd[0].data_ptr(), xd[1].data_ptr(),
                                xd[2].data_ptr() if cin == 3 else 0, Gd.data_ptr(), h.data_ptr(), scratch.data_ptr(),
                                scratch.numel(), gw.data_ptr(), gb.data_ptr(), s)
    Gt = r16(torch, G).permute(0, 3, 1, 2)
    (torch.relu(pre) * Gt).sum().backward()
    gxr = X.grad.numpy()
    gxr[:, 0] += 7.0                                                              # channel 0 accumulated
    assert rel(np.stack([t.cpu().numpy() for t in gx], 1), gxr) <= 1e-5
    gwr = Wt.grad.permute(2, 3, 1, 0).reshape(-1).numpy()                        # back to [tap][ci][co]
    assert rel(gw.cpu().numpy(), gwr) <= 1e-4
    assert rel(gb.cpu().numpy(), Bt.grad.numpy()) <= 1e-4
    # the fused call: both gradients in one pass, weight gradients accumulated onto the first ones
    gx2_ = [torch.full((B_, H_, W_), 7.0, device="cuda") for _ in range(cin)]
    pkg.tat_conv_in_bwd(B_, H_, W_, cin, xd[0].data_ptr(), xd[1].data_ptr(), xd[2].data_ptr() if cin == 3 else 0,
                        Gd.data_ptr(), h.data_ptr(), wd.data_ptr(), gx2_[0].data_ptr(), gx2_[1].data_ptr(),
                        gx2_[2].data_ptr() if cin == 3 else 0, 0b01, scratch.data_ptr(), scratch.numel(),
                        gw.data_ptr(), gb.data_ptr(), s)
    assert rel(np.stack([t.cpu().numpy() for t in gx2_], 1), gxr) <= 1e-5
    assert rel(gw.cpu().numpy(), 2 * gwr) <= 1e-4
    assert rel(gb.cpu().numpy(), 2 * Bt.grad.numpy()) <= 1e-4
    # pre-masked gradient (h = NULL): G * [h > 0] formed on the host
    Gm = dev_bf16(torch, (r16(torch, G) * (host_bf16(torch, h) > 0).to(torch.float64)).numpy())
    gx3 = [torch.full((B_, H_, W_), 7.0, device="cuda") for _ in range(cin)]
    pkg.tat_conv_in_bwd(B_, H_, W_, cin, xd[0].data_ptr(), xd[1].data_ptr(), xd[2].data_ptr() if cin == 3 else 0,
                        Gm.data_ptr(), 0, wd.data_ptr(), gx3[0].data_ptr(), gx3[1].data_ptr(),
                        gx3[2].data_ptr() if cin == 3 else 0, 0b01, scratch.data_ptr(), scratch.numel(),
                        gw.data_ptr(), gb.data_ptr(), s)
    assert rel(np.stack([t.cpu().numpy() for t in gx3], 1), gxr) <= 1e-5
    assert rel(gw.cpu().numpy(), 3 * gwr) <= 1e-4
    assert rel(gb.cpu().numpy(), 3 * Bt.grad.numpy()) <= 1e-4
    pkg.tat_lpd_check()


@pytest.mark.parametrize("size", LAYER_SIZES, ids=LAYER_IDS)
def test_conv_mid_forward_backward(pkg, torch, size):
    B_, H_, W_ = size
    import torch.nn.functional as F
    hin = np.maximum(gaussian(40, B_ * H_ * W_ * 32), 0).reshape(B_, H_, W_, 32)
    w = 0.08 * gaussian(41, 9 * 32 * 32)
    b = 0.05 * gaussian(42, 32)
    s = _stream(torch)
    hd, wd, bd = dev_bf16(torch, hin), dev_bf16(torch, w), dev32(torch, b)
    out = torch.empty_like(hd)
    pkg.tat_conv_mid_fwd(B_, H_, W_, hd.data_ptr(), wd.data_ptr(), bd.data_ptr(), out.data_ptr(), s)
    X = r16(torch, hin).permute(0, 3, 1, 2).contiguous().requires_grad_(True)
    Wt = r16(torch, w).reshape(3, 3, 32, 32).permute(2, 3, 0, 1).contiguous().requires_grad_(True)
    Bt = torch.tensor(np.asarray(b, np.float32), dtype=torch.float64).requires_grad_(True)
    pre = F.conv2d(X, Wt, Bt, padding=1)
    assert rel(host_bf16(torch, out).permute(0, 3, 1, 2), r16(torch, torch.relu(pre).detach())) <= 1e-3
    G = 0.5 * gaussian(43, B_ * H_ * W_ * 32).reshape(B_, H_, W_, 32)
    Gd = dev_bf16(torch, G)
    gin = torch.empty_like(hd)
    pkg.tat_conv_mid_bwd_data(B_, H_, W_, Gd.data_ptr(), out.data_ptr(), wd.data_ptr(), 0, gin.data_ptr(), s)
    scratch = torch.empty(pkg.tat_lpd_scratch_floats(B_, H_, W_), device="cuda")
    gw = torch.zeros(9 * 32 * 32, device="cuda")
    gb = torch.zeros(32, device="cuda")
    pkg.tat_conv_mid_bwd_weights(B_, H_, W_, hd.data_ptr(), Gd.data_ptr(), out.data_ptr(), scratch.data_ptr(),
                                 scratch.numel(), gw.data_ptr(), gb.data_ptr(), s)
    (torch.relu(pre) * r16(torch, G).permute(0, 3, 1, 2)).sum().backward()
    assert rel(host_bf16(torch, gin).permute(0, 3, 1, 2), r16(torch, X.grad)) <= 1e-3
    gwr = Wt.grad.permute(2, 3, 0, 1).reshape(-1).numpy()                                   # [tap][co][ci]
    assert rel(gw.cpu().numpy(), gwr) <= 1e-4
    assert rel(gb.cpu().numpy(), Bt.grad.numpy()) <= 1e-4
    # pre-masked gradient (h_out = NULL): G * [out > 0] formed on the host gives the same results
    outm = (host_bf16(torch, out) > 0).to(torch.float64)
    Gm = dev_bf16(torch, (r16(torch, G) * outm).numpy())
    gin2 = torch.empty_like(hd)
    pkg.tat_conv_mid_bwd_data(B_, H_, W_, Gm.data_ptr(), 0, wd.data_ptr(), 0, gin2.data_ptr(), s)
    gref = r16(torch, X.grad).permute(0, 2, 3, 1)                                       # NHWC
    assert rel(host_bf16(torch, gin2), gref) <= 1e-3
    # h_in: the result masked by [h_in > 0] (with the gradient's mask read in-kernel and pre-masked)
    inm = (host_bf16(torch, hd) > 0).to(torch.float64)
    for gsrc, hsrc in ((Gd, out), (Gm, None)):
        gin3 = torch.empty_like(hd)
        pkg.tat_conv_mid_bwd_data(B_, H_, W_, gsrc.data_ptr(), hsrc.data_ptr() if hsrc is not None else 0,
                                  wd.data_ptr(), hd.data_ptr(), gin3.data_ptr(), s)
        g3 = host_bf16(torch, gin3)
        assert rel(g3, gref * inm) <= 1e-3
        assert torch.all(g3[inm == 0] == 0)                                             # exactly zero where masked
    pkg.tat_conv_mid_bwd_weights(B_, H_, W_, hd.data_ptr(), Gm.data_ptr(), 0, scratch.data_ptr(), scratch.numel(),
                                 gw.data_ptr(), gb.data_ptr(), s)
    assert rel(gw.cpu().numpy(), 2 * gwr) <= 1e-4
    assert rel(gb.cpu().numpy(), 2 * Bt.grad.numpy()) <= 1e-4
    pkg.tat_lpd_check()     # no TMA tile wait gave up


@pytest.mark.parametrize("size", LAYER_SIZES, ids=LAYER_IDS)
def test_conv_out_forward_backward(pkg, torch, size):
    B_, H_, W_ = size
    import torch.nn.functional as F
    hin = np.maximum(gaussian(50, B_ * H_ * W_ * 32), 0).reshape(B_, H_, W_, 32)
    w = 0.1 * gaussian(51, 9 * 32)
    b = np.array([0.3])
    res = gaussian(52, B_ * H_ * W_).reshape(B_, H_, W_)
    s = _stream(torch)
    hd, wd, bd, rd = dev_bf16(torch, hin), dev_bf16(torch, w), dev32(torch, b), dev32(torch, res)
    out = torch.empty((B_, H_, W_), device="cuda")
    pkg.tat_conv_out_fwd(B_, H_, W_, hd.data_ptr(), wd.data_ptr(), bd.data_ptr(), rd.data_ptr(), out.data_ptr(), s)
    X = r16(torch, hin).permute(0, 3, 1, 2).contiguous().requires_grad_(True)
    Wt = r16(torch, w).reshape(3, 3, 32).permute(2, 0, 1).unsqueeze(0).contiguous().requires_grad_(True)
    Bt = torch.tensor(np.asarray(b, np.float32), dtype=torch.float64).requires_grad_(True)
    ref = torch.tensor(np.asarray(res, np.float32), dtype=torch.float64) + F.conv2d(X, Wt, Bt, padding=1)[:, 0]
    assert rel(out.cpu().numpy(), ref.detach().numpy()) <= 1e-5
    G = gaussian(53, B_ * H_ * W_).reshape(B_, H_, W_)
    Gd = dev32(torch, G)
    gh = torch.empty_like(hd)
    scratch = torch.empty(pkg.tat_lpd_scratch_floats(B_, H_, W_), device="cuda")
    gw = torch.zeros(9 * 32, device="cuda")
    gb = torch.zeros(1, device="cuda")
    pkg.tat_conv_out_bwd(B_, H_, W_, Gd.data_ptr(), hd.data_ptr(), wd.data_ptr(), 0, gh.data_ptr(),
                         scratch.data_ptr(), scratch.numel(), gw.data_ptr(), gb.data_ptr(), s)
    (ref * torch.tensor(np.asarray(G, np.float32), dtype=torch.float64)).sum().backward()
    assert rel(host_bf16(torch, gh).permute(0, 3, 1, 2), r16(torch, X.grad)) <= 1e-3
    assert rel(gw.cpu().numpy(), Wt.grad[0].permute(1, 2, 0).reshape(-1).numpy()) <= 1e-4
    assert rel(gb.cpu().numpy(), Bt.grad.numpy()) <= 1e-4
    # mask_relu: the same gradient times [h > 0] (h holds exact zeros where its ReLU clipped)
    ghm = torch.empty_like(hd)
    pkg.tat_conv_out_bwd(B_, H_, W_, Gd.data_ptr(), hd.data_ptr(), wd.data_ptr(), 1, ghm.data_ptr(),
                         scratch.data_ptr(), scratch.numel(), gw.data_ptr(), gb.data_ptr(), s)
    mask = (X > 0).to(torch.float64)
    assert rel(host_bf16(torch, ghm).permute(0, 3, 1, 2), r16(torch, X.grad) * mask) <= 1e-3
    assert rel(gw.cpu().numpy(), 2 * Wt.grad[0].permute(1, 2, 0).reshape(-1).numpy()) <= 1e-4
    pkg.tat_lpd_check()


def _problem(pkg, torch, n=32, B=2, seed=0):
    from oracle import solvers as S
    from oracle import tat_oracle as O
    op = pkg.TatOperator(n, 2 * n, 2 * n, device="cuda:0", support_radius=0.9)
    P = O.OraclePlan(n, 2 * n, 2 * n, support_radius=0.9)
    f = np.stack([ellipse_phantom(n, seed + b) for b in range(B)]).astype(np.float32)
    y = np.stack([O.forward(P, f[b].astype(np.float64)) for b in range(B)]).astype(np.float32)
    return op, S.plan_op(P), f, y


def test_lpd_loss_and_gradient_vs_oracle(pkg, torch):
    from oracle import lpd as OL
    op, oop, f, y = _problem(pkg, torch)
    _, npar = OL.layout()
    assert npar == pkg.lpd.NPARAM
    p = (0.1 * gaussian(60, npar)).astype(np.float32)
    net = pkg.lpd.LPD(op, 2, K=3, params=torch.tensor(p))
    loss, grad = net.loss_and_grad(dev32(torch, y), dev32(torch, f))
    lref, gref = OL.loss_and_grad(torch.tensor(p, dtype=torch.float64), oop, torch.tensor(y, dtype=torch.float64),
                                  torch.tensor(f, dtype=torch.float64), K=3, bf16=True)
    pkg.tat_lpd_check()
    assert abs(float(loss.item()) - lref) <= 2e-3 * lref
    assert rel(grad.cpu().numpy(), gref.numpy()) <= 2e-2
    fk = net.f[3].cpu().numpy()
    fref = OL.reconstruct(torch.tensor(p, dtype=torch.float64), oop, torch.tensor(y, dtype=torch.float64), 3, True)
    assert rel(fk, fref.detach().numpy()) <= 2e-3


def test_lpd_training_reduces_loss_and_graph_matches(pkg, torch):
    op, _, f, y = _problem(pkg, torch, n=32, B=4, seed=10)
    yd, fd = dev32(torch, y), dev32(torch, f)
    eager = pkg.lpd.LPD(op, 4, K=3, seed=1, lr=2e-3)
    graph = pkg.lpd.LPD(op, 4, K=3, seed=1, lr=2e-3)
    le, lg = [], []
    for _ in range(40):
        le.append(float(eager.train_step(yd, fd).item()))
        lg.append(float(graph.train_step(yd, fd, graph=True).item()))
    assert le[-1] < 0.5 * le[0] and lg[-1] < 0.5 * lg[0]
    # every kernel of the step adds in a fixed order (A*'s scatter included), so graph replay
    # and eager launches follow the same arithmetic over all 40 steps
    assert np.allclose(le, lg, rtol=1e-6, atol=0)


def test_lpd_graph_step_matches_eager_step_from_the_same_state(pkg, torch):
    """One training step at a time from identical states (parameters, BF16 copy, Adam moments,
    step count copied into the graph network first), for 40 steps: a replay bug that shows up
    only after some steps (a stale captured parameter, optimizer state) cannot hide behind
    differences that compound."""
    op, _, f, y = _problem(pkg, torch, n=32, B=4, seed=10)
    yd, fd = dev32(torch, y), dev32(torch, f)
    eager = pkg.lpd.LPD(op, 4, K=3, seed=1, lr=2e-3)
    graph = pkg.lpd.LPD(op, 4, K=3, seed=5, lr=2e-3)      # different initial weights on purpose
    for step in range(40):
        for name in ("params", "wbf", "m", "v"):
            getattr(graph, name).copy_(getattr(eager, name))
        graph.t = eager.t
        le = float(eager.train_step(yd, fd).item())
        lg = float(graph.train_step(yd, fd, graph=True).item())
        assert abs(le - lg) <= 1e-6 * abs(le), step
        pe, pg = eager.params.double(), graph.params.double()
        assert float((pe - pg).norm()) <= 1e-6 * float(pe.norm()), step


def test_trained_lpd_beats_tv_on_limited_view(pkg, torch):
    """What the learned part gains: trained on data from the fast A (512 phantoms, 2 % noise, detectors on a
    half circle), the LPD reconstruction error on held-out phantoms is below that of TV-LS on the same
    operators with its regularisation weight picked on the training data (Section 4.5 reports the same
    ordering for 180 degree data)."""
    import math as m
    from tat_inputs import add_noise, phantom_batch, roi_mask
    n, nd, nt, Bt = 64, 128, 128, 8
    op = pkg.TatOperator(n, nd, nt, device="cuda:0", support_radius=0.9, arc_begin=0.0, arc_len=m.pi)

    def data(seed0, count):
        f = torch.tensor(phantom_batch(n, count, seed0=seed0).astype(np.float32), device="cuda:0")
        g = op.forward(f).cpu().numpy()
        y = np.stack([add_noise(g[i], 0.02, seed0 + 5000 + i) for i in range(count)]).astype(np.float32)
        return f, torch.tensor(y, device="cuda:0")

    f_tr, y_tr = data(0, 512)
    f_te, y_te = data(20000, 8)
    net = pkg.lpd.LPD(op, Bt, K=10, seed=3, lr=1e-3)
    curve = net.fit(f_tr, y_tr, 2500, seed=1)
    assert curve[-1][1] < 0.2 * curve[0][1]

    def err(rec, ref):
        return float((torch.linalg.vector_norm((rec - ref).reshape(Bt, -1), dim=1) /
                      torch.linalg.vector_norm(ref.reshape(Bt, -1), dim=1)).mean())

    e_lpd = err(net.reconstruct(y_te).clone(), f_te)
    L = pkg.power_norm_sq(op, iters=40)
    sigma, tau, s = pkg.pdhg_steps(1.05 * L, op.info["h"])
    solver = pkg.TatSolver(op, Bt, mask=torch.tensor(roi_mask(n, radius=0.9), dtype=torch.float32, device="cuda:0"))
    alphas = (1e-5, 3e-5, 1e-4, 3e-4, 1e-3)
    tr_err = [err(solver.tv(y_tr[:Bt].contiguous(), a, 100, sigma, tau, s).clone(), f_tr[:Bt]) for a in alphas]
    a_best = alphas[int(np.argmin(tr_err))]
    e_tv = err(solver.tv(y_te, a_best, 100, sigma, tau, s).clone(), f_te)
    print(f"limited view, n=64: LPD {e_lpd:.4f}  TV-LS {e_tv:.4f} (alpha {a_best})")
    assert e_lpd < e_tv


def test_bounded_wait_gives_up_and_reports(pkg, torch):
    """A wait on an mbarrier that nothing arrives on runs out after its try count, sets the
    flag tat_lpd_check reports as TAT_ERR_TIMEOUT (once: the check clears it), and leaves the
    context usable: a convolution afterwards runs and matches the one before."""
    dev = torch.device("cuda:0")
    pkg.tat_lpd_check()                                   # start from a clear flag
    B_, H_, W_ = 1, 20, 36
    h = torch.from_numpy(np.abs(gaussian(60, B_ * H_ * W_ * 32)).astype(np.float32)).to(dev)
    hb = torch.empty(h.numel(), dtype=torch.int16, device=dev)
    pkg.tat_to_bf16(h.numel(), h.data_ptr(), hb.data_ptr())
    w = torch.from_numpy((0.05 * gaussian(61, 9 * 32 * 32)).astype(np.float32)).to(dev)
    wb = torch.empty(w.numel(), dtype=torch.int16, device=dev)
    pkg.tat_to_bf16(w.numel(), w.data_ptr(), wb.data_ptr())
    b = torch.zeros(32, dtype=torch.float32, device=dev)
    out0, out1 = torch.empty_like(hb), torch.empty_like(hb)
    pkg.tat_conv_mid_fwd(B_, H_, W_, hb.data_ptr(), wb.data_ptr(), b.data_ptr(), out0.data_ptr())
    gave_up = torch.zeros(1, dtype=torch.int32, device=dev)
    pkg.tat_lpd_timeout_probe(256, gave_up.data_ptr())
    torch.cuda.synchronize()
    assert int(gave_up.item()) == 1
    with pytest.raises(pkg.TatError) as err:
        pkg.tat_lpd_check()
    assert err.value.status == 5                          # TAT_ERR_TIMEOUT
    pkg.tat_lpd_check()                                   # cleared by the report
    pkg.tat_conv_mid_fwd(B_, H_, W_, hb.data_ptr(), wb.data_ptr(), b.data_ptr(), out1.data_ptr())
    torch.cuda.synchronize()
    assert torch.equal(out0, out1)
    pkg.tat_lpd_check()
