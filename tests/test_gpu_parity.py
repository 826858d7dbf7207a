"""GPU parity: libtat's CUDA path against the FP64 oracle, through the C ABI.

Bar: relative L2 error <= 1e-5 per image / per sinogram for FP32 device
arithmetic against the FP64 oracle on identical (FP32-representable) inputs.
"""
import math

import numpy as np
import pytest

from oracle import tat_oracle as O
from tat_inputs import ellipse_phantom, random_sinogram

pytestmark = pytest.mark.gpu

TOL = 1e-5


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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


CASES = {
    "n64": dict(n=64, n_det=128, n_t=128, support_radius=0.9),
    "n64_nolow": dict(n=64, n_det=128, n_t=128, support_radius=0.9, low_mode_quadrature=0),
    "n64_halfcircle": dict(n=64, n_det=128, n_t=128, support_radius=0.9, arc_begin=0.0, arc_len=math.pi),
    "n64_arc120": dict(n=64, n_det=128, n_t=128, support_radius=0.9, arc_begin=math.pi / 6, arc_len=2 * math.pi / 3),
    "n48_runtime_lengths": dict(n=48, n_det=96, n_t=100, support_radius=0.9),
    "n33_odd": dict(n=33, n_det=64, n_t=70, support_radius=0.98),
    "n64_fold": dict(n=64, n_det=64, n_t=128, support_radius=0.9, n_phi=256),
    "n64_physical": dict(n=64, n_det=128, n_t=128, support_radius=0.9, c=1.5, R=0.8, T=1.6),
    "n64_pad16": dict(n=64, n_det=128, n_t=128, support_radius=0.9, pad_L=16.0),
    # N = 8192: the four-step transform with a 32-point first step, in full (553 > 512 rows)
    # and pruned to two terms (440 <= 512 rows)
    "n553_N8192": dict(n=553, n_det=128, n_t=128, support_radius=0.9, T=6.0),
    "n440_N8192_pruned": dict(n=440, n_det=128, n_t=128, support_radius=0.9, T=8.0),
    # N = 4096: the column stages on the warp-split transform (n <= 512 rows; 220 rows leave
    # the upper half of every warp's inputs zero) and, with 586 rows (a smaller padding), on
    # the four-step one
    "n128_N1024": dict(n=128, n_det=128, n_t=128, support_radius=0.9),
    "n255_N2048": dict(n=255, n_det=128, n_t=128, support_radius=0.9),
    "n500_N4096_split": dict(n=500, n_det=128, n_t=128, support_radius=0.9),
    "n220_N4096_split": dict(n=220, n_det=128, n_t=128, support_radius=0.9, T=8.0),
    "n586_N4096_fourstep": dict(n=586, n_det=128, n_t=128, support_radius=0.9, pad_L=7.0),
}

_ORACLE_KEYS = {"low_mode_quadrature": "low_mode"}


def make(pkg, torch, kw):
    desc = dict(kw)
    n, nd, nt = desc.pop("n"), desc.pop("n_det"), desc.pop("n_t")
    c, R, T = desc.pop("c", 1.0), desc.pop("R", 1.0), desc.pop("T", 2.0)
    op = pkg.TatOperator(n, nd, nt, c=c, R=R, T=T, device="cuda:0", **desc)
    okw = {_ORACLE_KEYS.get(k, k): (bool(v) if k == "low_mode_quadrature" else v) for k, v in desc.items()}
    P = O.OraclePlan(n, nd, nt, c=c, R=R, T=T, **okw)
    return op, P


@pytest.mark.parametrize("name", list(CASES))
def test_forward_parity(pkg, torch, name):
    op, P = make(pkg, torch, CASES[name])
    f = f32(ellipse_phantom(P.n, 0))
    g = op.forward(torch.tensor(f, dtype=torch.float32, device="cuda:0")).cpu().numpy()
    ref = O.forward(P, f)
    assert g.shape == (P.n_det, P.n_t)
    assert rel(g, ref) <= TOL


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_parity(pkg, torch, name):
    op, P = make(pkg, torch, CASES[name])
    gin = f32(random_sinogram(P.n_det, P.n_t, 1))
    f = op.adjoint(torch.tensor(gin, dtype=torch.float32, device="cuda:0")).cpu().numpy()
    ref = O.adjoint(P, gin)
    assert f.shape == (P.n, P.n)
    assert rel(f, ref) <= TOL


@pytest.mark.parametrize("name", ["n64", "n128_N1024", "n255_N2048", "n500_N4096_split", "n220_N4096_split",
                                  "n553_N8192", "n440_N8192_pruned"])
def test_column_split_variants(pkg, torch, name):
    """At N = 512 RB (RB = 1 .. 16) with at most 512 rows (1024 at N = 8192) either column
    stage runs on the warp-split transform or on the four-step one (a bit each in the
    plan's mask): both against the oracle and each other, batch 3; each stage's result
    depends only on its own bit, bit for bit; the split A* the same bits on repeated calls
    and for other column strips."""
    op, P = make(pkg, torch, CASES[name])
    N = op.info["N"]
    assert pkg.tat_plan_get_column_split(op.plan) == {512: 1, 8192: 2}.get(N, 3)
    B = 3
    fs = np.stack([f32(ellipse_phantom(P.n, 70 + s)) for s in range(B)])
    gs = np.stack([f32(random_sinogram(P.n_det, P.n_t, 80 + s)) for s in range(B)])
    ft = torch.tensor(fs, dtype=torch.float32, device="cuda:0")
    gt = torch.tensor(gs, dtype=torch.float32, device="cuda:0")
    out = {}
    for mask in (3, 0, 1, 2):
        pkg.tat_plan_set_column_split(op.plan, mask)
        assert pkg.tat_plan_get_column_split(op.plan) == mask
        out[mask] = (op.forward(ft).cpu().numpy(), op.adjoint(gt).cpu().numpy())
    g_split, fa_split = out[3]
    g_four, fa_four = out[0]
    assert np.array_equal(out[1][0], g_split) and np.array_equal(out[1][1], fa_four)
    assert np.array_equal(out[2][0], g_four) and np.array_equal(out[2][1], fa_split)
    pkg.tat_plan_set_column_split(op.plan, 3)
    assert np.array_equal(op.adjoint(gt).cpu().numpy(), fa_split)
    big = N == 8192                                             # one row pair, 512-thread CTAs there
    pkg.tat_plan_set_launch_shape(op.plan, 3, 1 if big else 2, 512 if big else 256, 0)   # strips of 3 columns
    assert np.array_equal(op.adjoint(gt).cpu().numpy(), fa_split)
    assert np.array_equal(op.forward(ft).cpu().numpy(), g_split)
    for s in (0, B - 1):
        assert rel(g_split[s], O.forward(P, fs[s])) <= TOL
        assert rel(fa_split[s], O.adjoint(P, gs[s])) <= TOL
        assert rel(g_four[s], g_split[s].astype(np.float64)) <= 1e-6
        assert rel(fa_four[s], fa_split[s].astype(np.float64)) <= 1e-6
    with pytest.raises(pkg.TatError):
        pkg.tat_plan_set_column_split(op.plan, 4)


def test_plan_matches_oracle_grid(pkg, torch):
    op, P = make(pkg, torch, CASES["n64"])
    info = op.info
    assert (info["N"], info["M"], info["J"], info["n_phi"]) == (P.N, P.M, P.J, P.n_phi)


def test_dot_product_fp32(pkg, torch):
    """<A f, g>_Y = <f, A* g>_X with both sides computed by the CUDA path."""
    op, P = make(pkg, torch, CASES["n64"])
    f = f32(ellipse_phantom(64, 3))
    g = f32(random_sinogram(128, 128, 4))
    Af = op.forward(torch.tensor(f, dtype=torch.float32, device="cuda:0")).cpu().numpy().astype(np.float64)
    Asg = op.adjoint(torch.tensor(g, dtype=torch.float32, device="cuda:0")).cpu().numpy().astype(np.float64)
    lhs = P.W_Y * np.sum(Af * g)
    rhs = P.W_X * np.sum(f * Asg)
    # normalised by the Cauchy-Schwarz bound of both sides
    scale = max(P.W_Y * np.linalg.norm(Af) * np.linalg.norm(g), P.W_X * np.linalg.norm(f) * np.linalg.norm(Asg))
    assert abs(lhs - rhs) <= 1e-5 * scale


def test_batched_equals_single_and_strides(pkg, torch):
    op, P = make(pkg, torch, CASES["n64"])
    B = 5
    fs = np.stack([f32(ellipse_phantom(64, s)) for s in range(B)])
    # padded stride between images
    pad = np.zeros((B, 64 * 64 + 37), np.float32)
    pad[:, : 64 * 64] = fs.reshape(B, -1)
    fpad = torch.tensor(pad, device="cuda:0")
    g = torch.empty((B, 128 * 128 + 5), dtype=torch.float32, device="cuda:0")
    ws = op.workspace(B)
    pkg.tat_forward_batched(op.plan, B, fpad.data_ptr(), pad.shape[1], g.data_ptr(), g.shape[1], ws.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    gb = g[:, : 128 * 128].reshape(B, 128, 128).cpu().numpy()
    for s in range(B):
        single = op.forward(torch.tensor(fs[s], dtype=torch.float32, device="cuda:0")).cpu().numpy()
        assert np.array_equal(gb[s], single)
        assert rel(gb[s], O.forward(P, fs[s])) <= TOL
    gs = np.stack([f32(random_sinogram(128, 128, 10 + s)) for s in range(B)])
    fa = op.adjoint(torch.tensor(gs, dtype=torch.float32, device="cuda:0")).cpu().numpy()
    for s in (0, B - 1):
        assert rel(fa[s], O.adjoint(P, gs[s])) <= TOL


def test_batched_strides_split_columns(pkg, torch):
    """Batched A and A* with padded image and sinogram strides through the warp-split column
    stages (n = 500, N = 4096, odd batch 3): every image equals its single-image call bit for
    bit, and the last one matches the oracle."""
    op, P = make(pkg, torch, CASES["n500_N4096_split"])
    assert pkg.tat_plan_get_column_split(op.plan) == 3
    n, nd, nt, B = P.n, P.n_det, P.n_t, 3
    fs = np.stack([f32(ellipse_phantom(n, 20 + s)) for s in range(B)])
    fpad = np.zeros((B, n * n + 6), np.float32)
    fpad[:, : n * n] = fs.reshape(B, -1)
    fp = torch.tensor(fpad, device="cuda:0")
    g = torch.empty((B, nd * nt + 10), dtype=torch.float32, device="cuda:0")
    ws = op.workspace(B)
    st = torch.cuda.current_stream().cuda_stream
    pkg.tat_forward_batched(op.plan, B, fp.data_ptr(), fpad.shape[1], g.data_ptr(), g.shape[1], ws.data_ptr(), st)
    gb = g[:, : nd * nt].reshape(B, nd, nt).cpu().numpy()
    for s in range(B):
        single = op.forward(torch.tensor(fs[s], dtype=torch.float32, device="cuda:0")).cpu().numpy()
        assert np.array_equal(gb[s], single)
    assert rel(gb[B - 1], O.forward(P, fs[B - 1])) <= TOL
    gs = np.stack([f32(random_sinogram(nd, nt, 30 + s)) for s in range(B)])
    gpad = np.zeros((B, nd * nt + 10), np.float32)
    gpad[:, : nd * nt] = gs.reshape(B, -1)
    gp = torch.tensor(gpad, device="cuda:0")
    fo = torch.empty((B, n * n + 6), dtype=torch.float32, device="cuda:0")
    pkg.tat_adjoint_batched(op.plan, B, gp.data_ptr(), gpad.shape[1], fo.data_ptr(), fo.shape[1], ws.data_ptr(), st)
    fb = fo[:, : n * n].reshape(B, n, n).cpu().numpy()
    for s in range(B):
        single = op.adjoint(torch.tensor(gs[s], dtype=torch.float32, device="cuda:0")).cpu().numpy()
        assert np.array_equal(fb[s], single)
    assert rel(fb[B - 1], O.adjoint(P, gs[B - 1])) <= TOL


def test_zero_input_and_determinism(pkg, torch):
    op, P = make(pkg, torch, CASES["n64"])
    z = torch.zeros((2, 64, 64), dtype=torch.float32, device="cuda:0")
    assert float(op.forward(z).abs().max()) == 0.0
    zg = torch.zeros((2, 128, 128), dtype=torch.float32, device="cuda:0")
    assert float(op.adjoint(zg).abs().max()) == 0.0
    f = torch.tensor(f32(ellipse_phantom(64, 9)), dtype=torch.float32, device="cuda:0")
    a, b = op.forward(f), op.forward(f)
    assert torch.equal(a, b)
    # A* too: its scatter adds in a fixed order (no atomics), so repeated calls agree bit for bit
    g = torch.tensor(f32(random_sinogram(128, 128, 9)), dtype=torch.float32, device="cuda:0").expand(3, 128, 128)
    fa, fb = op.adjoint(g.contiguous()), op.adjoint(g.contiguous())
    assert torch.equal(fa, fb)
    assert torch.equal(fa[0], fa[2])


def test_invalid_arguments(pkg, torch):
    op, P = make(pkg, torch, CASES["n64"])
    f = torch.zeros((64, 64), dtype=torch.float32, device="cuda:0")
    g = torch.zeros((128, 128), dtype=torch.float32, device="cuda:0")
    ws = op.workspace(1)
    st = torch.cuda.current_stream().cuda_stream
    with pytest.raises(pkg.TatError) as e:
        pkg.tat_forward(op.plan, f.data_ptr(), g.data_ptr(), 0, st)
    assert e.value.status == 1
    with pytest.raises(pkg.TatError):
        pkg.tat_forward(op.plan, f.data_ptr(), g.data_ptr(), ws.data_ptr() + 4, st)   # misaligned workspace
    with pytest.raises(pkg.TatError):
        pkg.tat_forward_batched(op.plan, 1, f.data_ptr(), 100, g.data_ptr(), 128 * 128, ws.data_ptr(), st)
    with pytest.raises(pkg.TatError):
        pkg.tat_forward_batched(op.plan, 0, f.data_ptr(), 64 * 64, g.data_ptr(), 128 * 128, ws.data_ptr(), st)


def test_n256_batch32_sampled(pkg, torch):
    """Batched workload n=256, 512 detectors x 512 samples, B=32 with the launch shapes the
    autotuner picks (as the benchmark runs it): images 0 and 31 against the oracle."""
    op, P = make(pkg, torch, dict(n=256, n_det=512, n_t=512, support_radius=0.9))
    B = 32
    op.autotune(B)
    fs = np.stack([f32(ellipse_phantom(256, s)) for s in range(B)])
    g = op.forward(torch.tensor(fs, dtype=torch.float32, device="cuda:0")).cpu().numpy()
    for s in (0, B - 1):
        assert rel(g[s], O.forward(P, fs[s])) <= TOL
    gs = np.stack([f32(random_sinogram(512, 512, 100 + s)) for s in (0, 1)])
    gi = torch.zeros((B, 512, 512), dtype=torch.float32, device="cuda:0")
    gi[0] = torch.tensor(gs[0], device="cuda:0")
    gi[B - 1] = torch.tensor(gs[1], device="cuda:0")
    fa = op.adjoint(gi).cpu().numpy()
    assert rel(fa[0], O.adjoint(P, gs[0])) <= TOL
    assert rel(fa[B - 1], O.adjoint(P, gs[1])) <= TOL
    assert float(np.abs(fa[1:B - 1]).max()) == 0.0


def test_headline_n512_full(pkg, torch):
    """n=512, 1024 detectors x 1024 samples, in the launch the benchmark times: B=32 with the
    autotuned launch shapes; images 0 and 31 of A and two images of A* against the oracle."""
    op, P = make(pkg, torch, dict(n=512, n_det=1024, n_t=1024, support_radius=0.9))
    B = 32
    op.autotune(B)
    fs = np.stack([f32(ellipse_phantom(512, s)) for s in range(B)])
    g = op.forward(torch.tensor(fs, dtype=torch.float32, device="cuda:0")).cpu().numpy()
    for s in (0, B - 1):
        assert rel(g[s], O.forward(P, fs[s])) <= TOL
    gins = [f32(random_sinogram(1024, 1024, 5 + s)) for s in (0, 1)]
    gi = torch.zeros((B, 1024, 1024), dtype=torch.float32, device="cuda:0")
    gi[1] = torch.tensor(gins[0], device="cuda:0")
    gi[B - 2] = torch.tensor(gins[1], device="cuda:0")
    fa_dev = op.adjoint(gi)
    fa = fa_dev.cpu().numpy()
    assert rel(fa[1], O.adjoint(P, gins[0])) <= TOL
    assert rel(fa[B - 2], O.adjoint(P, gins[1])) <= TOL
    # a second call of the full batch gives the same bits (the scatter has a fixed order of additions)
    assert torch.equal(op.adjoint(gi), fa_dev)


@pytest.mark.parametrize("n,cols_threads,strip,row_threads,row_pairs",
                         [(128, 64, 4, 64, 8), (128, 128, 16, 128, 4), (256, 64, 2, 0, 1), (256, 128, 8, 0, 2)])
def test_small_column_ctas(pkg, torch, n, cols_threads, strip, row_threads, row_pairs):
    """Column CTAs of 64 and 128 threads and row groups of 64 and 128 threads (the four-step
    FFTs of N = 8n on fewer threads than 256) against the oracle, batch 3, and the forward
    bit-identical to the default shape."""
    op, P = make(pkg, torch, dict(n=n, n_det=2 * n, n_t=2 * n, support_radius=0.9))
    pkg.tat_plan_set_column_split(op.plan, 0)   # the four-step column transform, whose CTA size varies
    B = 3
    fs = np.stack([f32(ellipse_phantom(n, 40 + s)) for s in range(B)])
    ft = torch.tensor(fs, dtype=torch.float32, device="cuda:0")
    g_default = op.forward(ft).cpu().numpy()
    inv_default = op.inverse(torch.tensor(g_default, device="cuda:0")).cpu().numpy()
    gs0 = np.stack([f32(random_sinogram(2 * n, 2 * n, 60 + s)) for s in range(B)])
    fa_default = op.adjoint(torch.tensor(gs0, dtype=torch.float32, device="cuda:0")).cpu().numpy()
    pkg.tat_plan_set_launch_shape(op.plan, strip, row_pairs, cols_threads, row_threads)
    g = op.forward(ft).cpu().numpy()
    assert np.array_equal(g, g_default)
    for s in range(B):
        assert rel(g[s], O.forward(P, fs[s])) <= TOL
    gs = np.stack([f32(random_sinogram(2 * n, 2 * n, 60 + s)) for s in range(B)])
    fa = op.adjoint(torch.tensor(gs, dtype=torch.float32, device="cuda:0")).cpu().numpy()
    for s in range(B):
        assert rel(fa[s], O.adjoint(P, gs[s])) <= TOL
    assert np.array_equal(fa, fa_default)   # each run of the scatter is summed the same way in any CTA shape
    inv = op.inverse(torch.tensor(g_default, device="cuda:0")).cpu().numpy()   # the inverse's column stage too
    assert rel(inv, inv_default) <= 1e-6


@pytest.mark.parametrize("n", [64, 256])
def test_fft_pass_order_variant(pkg, torch, n):
    """The other pass order of the length-2M FFT in the cosine and sine stages (the autotuner's
    FFT choice): A, A* and A^-1 against the oracle at the parity bar, and against order 0."""
    op, P = make(pkg, torch, dict(n=n, n_det=2 * n, n_t=2 * n, support_radius=0.9))
    B = 2
    fs = np.stack([f32(ellipse_phantom(n, 70 + s)) for s in range(B)])
    gs = np.stack([f32(random_sinogram(2 * n, 2 * n, 80 + s)) for s in range(B)])
    ft = torch.tensor(fs, dtype=torch.float32, device="cuda:0")
    gt = torch.tensor(gs, dtype=torch.float32, device="cuda:0")
    ref = {name: getattr(op, name)(x).cpu().numpy() for name, x in (("forward", ft), ("adjoint", gt), ("inverse", gt))}
    assert pkg.tat_plan_get_fft_order(op.plan) == 0
    pkg.tat_plan_set_fft_order(op.plan, 1)
    assert pkg.tat_plan_get_fft_order(op.plan) == 1
    out = {name: getattr(op, name)(x).cpu().numpy() for name, x in (("forward", ft), ("adjoint", gt), ("inverse", gt))}
    for s_ in range(B):
        assert rel(out["forward"][s_], O.forward(P, fs[s_])) <= TOL
        assert rel(out["adjoint"][s_], O.adjoint(P, gs[s_])) <= TOL
    assert rel(out["inverse"][0], O.inverse(P, gs[0])) <= TOL
    for name in out:
        assert rel(out[name], ref[name]) <= 1e-6
    with pytest.raises(pkg.TatError):
        pkg.tat_plan_set_fft_order(op.plan, 2)
    pkg.tat_plan_set_fft_order(op.plan, 0)

