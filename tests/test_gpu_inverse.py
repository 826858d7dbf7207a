"""GPU parity of the approximate inverse A^{-1} (Algorithm 3) against the FP64 oracle.

Bar: relative L2 error <= 1e-5 per image, FP32 device arithmetic against the
FP64 oracle on identical FP32-representable data, through the C ABI.
"""
import math

import numpy as np
import pytest

from oracle import tat_oracle as O
from tat_inputs import add_noise, ellipse_phantom, random_sinogram

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
    "n64_T4": dict(n=64, n_det=128, n_t=128, support_radius=0.98, T=4.0),
    "n64_halfcircle": dict(n=64, n_det=128, n_t=128, support_radius=0.9, arc_begin=0.0, arc_len=math.pi),
    "n48_runtime_lengths": dict(n=48, n_det=96, n_t=100, support_radius=0.9),
    "n33_odd": dict(n=33, n_det=64, n_t=70, support_radius=0.98),
    "n64_physical": dict(n=64, n_det=128, n_t=128, support_radius=0.9, c=1.5, R=0.8, T=1.6),
    "n128": dict(n=128, n_det=256, n_t=256, support_radius=0.9),
}


def make(pkg, kw):
    desc = dict(kw)
    n, nd, nt = desc.pop("n"), desc.pop("n_det"), desc.pop("n_t")
    c, R, T = desc.pop("c", 1.0), desc.pop("R", 1.0), desc.pop("T", 2.0)
    op = pkg.TatOperator(n, nd, nt, c=c, R=R, T=T, device="cuda:0", **desc)
    P = O.OraclePlan(n, nd, nt, c=c, R=R, T=T, **desc)
    return op, P


@pytest.mark.parametrize("name", list(CASES))
def test_inverse_parity_random_data(pkg, torch, name):
    op, P = make(pkg, CASES[name])
    g = f32(random_sinogram(P.n_det, P.n_t, 11))
    fd = op.inverse(torch.tensor(g, dtype=torch.float32, device="cuda:0")).cpu().numpy()
    ref = O.inverse(P, g)
    assert fd.shape == (P.n, P.n)
    assert rel(fd, ref) <= TOL
    assert np.all(fd[P.mask == 0] == 0)


@pytest.mark.parametrize("name", ["n64", "n64_T4", "n64_halfcircle"])
def test_inverse_parity_phantom_data(pkg, torch, name):
    op, P = make(pkg, CASES[name])
    g = f32(add_noise(O.forward(P, ellipse_phantom(P.n, 2)), 0.01, 3))
    fd = op.inverse(torch.tensor(g, dtype=torch.float32, device="cuda:0")).cpu().numpy()
    assert rel(fd, O.inverse(P, g)) <= TOL


def test_left_inverse_on_device(pkg, torch):
    """A^{-1} A f = f to 0.3 % for a smooth bump with T = 4 on the full circle, both on the GPU."""
    op, P = make(pkg, CASES["n64_T4"])
    x = -1 + P.h * np.arange(P.n)
    X, Y = np.meshgrid(x, x)
    f = (np.exp(-((X - 0.2) ** 2 + (Y + 0.1) ** 2) / (2 * 0.15 ** 2)) * P.mask).astype(np.float32)
    ft = torch.tensor(f, device="cuda:0")
    fr = op.inverse(op.forward(ft)).cpu().numpy()
    assert rel(fr, f.astype(np.float64)) < 3e-3


def test_inverse_repeats_bit_for_bit(pkg, torch):
    """Repeated A^-1 calls give the same bits: the constant C is summed from per-CTA partial
    sums in a fixed order (no atomics), at a size with many row CTAs."""
    op, P = make(pkg, dict(n=500, n_det=128, n_t=128, support_radius=0.9))
    g = np.stack([f32(random_sinogram(128, 128, 70 + s)) for s in range(2)]).astype(np.float32)
    gt = torch.tensor(g, device="cuda:0")
    a = op.inverse(gt).cpu().numpy()
    assert np.array_equal(op.inverse(gt).cpu().numpy(), a)
    assert rel(a[1], O.inverse(P, g[1].astype(np.float64))) <= TOL


def test_inverse_batched_matches_single(pkg, torch):
    op, P = make(pkg, CASES["n64"])
    gs = np.stack([f32(random_sinogram(P.n_det, P.n_t, 20 + b)) for b in range(3)]).astype(np.float32)
    fb = op.inverse(torch.tensor(gs, device="cuda:0")).cpu().numpy()
    for b in range(3):
        f1 = op.inverse(torch.tensor(gs[b], device="cuda:0")).cpu().numpy()
        assert rel(fb[b], f1) <= 1e-6


def test_inverse_requires_own_angular_grid(pkg, torch):
    op = pkg.TatOperator(64, 64, 128, device="cuda:0", support_radius=0.9, n_phi=256)
    with pytest.raises(pkg.TatError):
        op.inverse(torch.zeros((64, 128), device="cuda:0"))


def test_inverse_headline_size(pkg, torch):
    """n = 512, 1024 detectors x 1024 samples, batch of 2: image 1 against the oracle."""
    op, P = make(pkg, dict(n=512, n_det=1024, n_t=1024, support_radius=0.9))
    g1 = f32(add_noise(O.forward(P, ellipse_phantom(512, 9)), 0.01, 10))
    g = np.stack([f32(random_sinogram(1024, 1024, 12)), g1]).astype(np.float32)
    fd = op.inverse(torch.tensor(g, device="cuda:0")).cpu().numpy()
    assert rel(fd[1], O.inverse(P, g1)) <= TOL
