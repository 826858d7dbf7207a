"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a direct sum,
a closed form, the Green's-function formula of the paper, the unaccelerated
Fourier method the paper uses for its own accuracy check, an exact transpose
built from dense matrices, or an exact symmetry of the discretisation.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss
from scipy.integrate import quad
from scipy.special import dawsn, j0

from oracle import tat_oracle as O
from tat_inputs import ellipse_phantom, random_sinogram


def _dense(P, fn, shape_in):
    size = int(np.prod(shape_in))
    cols = [fn(P, np.eye(size)[i].reshape(shape_in)).ravel() for i in range(size)]
    return np.stack(cols, axis=1)


# ------------------------------------------------------------ plan integers

@pytest.mark.parametrize("n,nd,nt,N,M,J1", [
    (64, 128, 128, 512, 384, 190),        # n=64 parity workload
    (128, 256, 256, 1024, 768, 382),      # n=128 learned primal-dual workload
    (256, 512, 512, 2048, 1536, 766),     # n=256 batched workload
    (512, 1024, 1024, 4096, 3072, 1534),  # n=512 headline workload
    (1024, 2048, 2048, 8192, 6144, 3070), # n=1024 service member
])
def test_plan_integers(n, nd, nt, N, M, J1):
    """Grid rules of Section 3.1: T_new = max(2T,6), L = T_new + 2, lambda_j = j*pi/T_new."""
    P = O.OraclePlan(n, nd, nt, T=2.0)
    assert (P.N, P.M, P.J + 1, P.n_phi) == (N, M, J1, nd)
    assert P.T_ext >= 6.0 and P.L >= P.T_ext + 2.0 - 1e-12
    # no bilinear stencil reaches the unpaired Nyquist row/column
    assert P.lam[-1] / P.dxi < P.N / 2 - 1


def test_smooth_ceil():
    assert O.smooth_ceil(381.0) == 384
    assert O.smooth_ceil(384.0) == 384
    assert O.smooth_ceil(385.0) == 432
    assert O.smooth_ceil(2100.0) == 2187
    assert O.smooth_ceil(2100.0, even=True) == 2304


# ------------------------------------------------------------ single steps

def test_spectrum_matches_direct_dtft():
    """Step 2 against the direct sum (h^2/2pi) sum_x f(x) e^{-i xi.x} (Section 2.1 convention)."""
    P = O.OraclePlan(12, 16, 16, support_radius=1.5)
    rng = np.random.default_rng(1)
    f = rng.standard_normal((12, 12))
    F = O.spectrum(P, f)
    x = -1.0 + np.arange(12) * P.h
    for qx, qy in [(0, 0), (3, -5), (-P.N // 2 + 1, 7), (P.N // 2 - 1, P.N // 2 - 1), (17, -31)]:
        e = np.exp(-1j * (qx * P.dxi * x[None, :] + qy * P.dxi * x[:, None]))
        ref = P.h ** 2 / (2 * math.pi) * np.sum(f * e)
        assert abs(F[qy % P.N, qx % P.N] - ref) <= 1e-13 * np.abs(f).sum()


def test_bilinear_exact_on_affine():
    """Step 3 reproduces any function affine in (xi_x, xi_y) exactly."""
    P = O.OraclePlan(16, 32, 32)
    q = np.fft.fftfreq(P.N, 1.0 / P.N)
    QX, QY = np.meshgrid(q, q, indexing="xy")
    al, be, ga = 0.3 - 1.1j, 0.7 + 0.2j, -0.4 + 0.9j
    F = al + be * QX + ga * QY
    Fp = O.polar(P, F, P.lam)
    ref = al + (be * np.cos(P.phi)[None, :] + ga * np.sin(P.phi)[None, :]) * P.lam[:, None] / P.dxi
    assert np.abs(Fp - ref).max() <= 1e-12 * np.abs(ref).max()


def test_modes_pick_single_harmonic():
    """Step 4 (Eq. eq3): a ring equal to e^{i k0 phi} has one nonzero coefficient, at k0."""
    P = O.OraclePlan(16, 32, 32)
    for k0 in (0, 1, -1, 5, -16):
        Fp = np.exp(1j * k0 * P.phi)[None, :] * np.ones((3, 1))
        fh = O.modes(P, Fp)
        b = int(np.nonzero(P.k == k0)[0][0])
        assert abs(fh[1, b] - 1.0) < 1e-13
        fh[:, b] = 0
        assert np.abs(fh).max() < 1e-13


def test_bessel_table_jacobi_anger():
    """Eq. Anger: sum_k i^|k| J_|k|(lam) e^{ik theta} = e^{i lam cos theta} over the plan's mode bins."""
    P = O.OraclePlan(32, 128, 64)       # modes |k| <= 64: the series is converged for lam <= 17
    lam = np.array([0.0, 0.7, 5.3, 17.0])
    Jt = O.bessel_table(P, lam)                         # (4, n_phi)
    th = np.linspace(0, 2 * math.pi, 13)
    lhs = (Jt * (1j) ** P.absk[None, :]) @ np.exp(1j * P.k[:, None] * th[None, :])
    assert np.abs(lhs - np.exp(1j * lam[:, None] * np.cos(th)[None, :])).max() < 1e-13


def test_hybrid_rule_moments():
    """Low-mode rule: exact on polynomials in the Euler-Maclaurin sense, nodes inside (0, a)."""
    x, w = O.hybrid_rule()
    a = O.LOW_A
    assert x.min() > 0 and x.max() < a and x.min() < 0.05 * a   # clustered toward 0
    # q(x) = (x - a)^p e^{...} is not polynomial; use truncated exact integrals instead:
    # int_0^inf e^{-s x} dx = 1/s is reproduced by the rule to high order for small s.
    for s in (0.05, 0.2, 0.5):
        j = np.arange(a, 4000)
        approx = np.sum(w * np.exp(-s * x)) + np.sum(np.exp(-s * j))
        assert abs(approx - 1.0 / s) < 1e-9 / s


@pytest.mark.parametrize("b,t", [(0.0025, 0.0), (0.01, 0.5), (0.05, 1.0), (0.2, 2.0)])
def test_hybrid_rule_dawson(b, t):
    """int_0^inf lam e^{-b lam^2} cos(lam t) dlam = (1 - 2 s D(s)) / (2b), s = t/(2 sqrt b)."""
    P = O.OraclePlan(64, 128, 128)
    x, w = O.hybrid_rule()
    h = P.dlam
    fn = lambda lam: lam * np.exp(-b * lam ** 2) * np.cos(lam * t)
    j = np.arange(O.LOW_A, 20000)
    approx = h * (np.sum(w * fn(x * h)) + np.sum(fn(j * h)))
    s = t / (2 * math.sqrt(b))
    exact = (1 - 2 * s * dawsn(s)) / (2 * b)
    trap = h * np.sum(fn(np.arange(1, 20000) * h))
    assert abs(approx - exact) < 1e-7
    assert abs(trap - exact) > 1e-2     # the plain trapezoid sum is far off


# ------------------------------------------------------------ adjoint

@pytest.mark.parametrize("kw", [
    {},
    {"low_mode": False},
    {"arc_begin": 0.0, "arc_len": math.pi},
    {"n_phi": 32},
    {"c": 1.5, "R": 0.8, "T": 1.6},
])
def test_adjoint_is_exact_transpose(kw):
    """A* = W_X^{-1} A^T W_Y with the inner products of Eq. innerProducts (dense matrices, n = 8)."""
    base = dict(n=8, n_det=16, n_t=16, support_radius=0.9)
    base.update(kw)
    P = O.OraclePlan(**base)
    A = _dense(P, O.forward, (8, 8))
    As = _dense(P, O.adjoint, (16, 16))
    ref = (A.T * P.W_Y) / P.W_X
    assert np.abs(As - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(A).max() > 1e-3


def test_dot_product():
    """<A f, g>_Y = <f, A* g>_X (Eq. innerProducts) on a random-ellipse phantom, n = 32."""
    P = O.OraclePlan(32, 64, 64, support_radius=0.9)
    f = ellipse_phantom(32, 3)
    g = random_sinogram(64, 64, 7)
    lhs = P.W_Y * np.sum(O.forward(P, f) * g)
    rhs = P.W_X * np.sum(f * O.adjoint(P, g))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ------------------------------------------------------------ against continuous truth

def _gauss_closed(sig, t):
    fn = lambda l: l * (sig ** 2 / 2) * np.exp(-sig ** 2 * l ** 2 / 4) * j0(l) * np.cos(l * t)
    return quad(fn, 0, 60 / sig, limit=2000, epsabs=1e-13)[0]


def test_centred_gaussian_closed_form():
    """f = exp(-|x|^2/s^2): fhat = (s^2/2)e^{-s^2 lam^2/4}, only k = 0 survives (Eq. eq2)."""
    sig = 0.12
    errs = {}
    for low in (True, False):
        P = O.OraclePlan(64, 128, 128, low_mode=low)
        x = -1 + np.arange(64) * P.h
        X, Y = np.meshgrid(x, x)
        g = O.forward(P, np.exp(-(X ** 2 + Y ** 2) / sig ** 2))
        ref = np.array([_gauss_closed(sig, t) for t in P.t])
        errs[low] = np.linalg.norm(g - ref[None, :]) / (np.linalg.norm(ref) * math.sqrt(128))
        if low:
            assert np.abs(g - g[:1]).max() <= 1e-4 * np.abs(g).max()   # theta-independent
    assert errs[True] < 5e-4
    assert errs[False] > 10 * errs[True]       # the low-mode quadrature is what makes it accurate


# ------------------------------------------------------------ physical units (c, R != 1)
#
# Section 2.1 sets R = c = 1 "without loss of generality"; the oracle takes
# physical (c, R, T) and normalises internally.  These pins state the physical
# problem on their own: the wave equation p_tt = c^2 Lap p with p(0) = f,
# p_t(0) = 0 on a grid of n nodes over [-R, R]^2, detectors on |z| = R at
# t_m = m T/(n_t - 1), and the L2 inner products of Eq. innerProducts in
# physical units (dx on the plane, arc length R dtheta times dt on the data).

_PHYS = dict(c=1.5, R=0.8, T=1.6)


def _gauss_physical(sig, c, R, t):
    """p(z, t) at |z| = R for f = exp(-|x|^2/sig^2), all in physical units.

    Radial Fourier synthesis of the wave equation: p = int_0^inf lam fhat(lam)
    J_0(lam R) cos(c lam t) dlam with fhat(lam) = (sig^2/2) exp(-sig^2 lam^2/4).
    """
    fn = lambda l: l * (sig ** 2 / 2) * np.exp(-sig ** 2 * l ** 2 / 4) * j0(l * R) * np.cos(c * l * t)
    return quad(fn, 0, 60 / sig, limit=2000, epsabs=1e-13)[0]


def _physical_gaussian_error(P, c, R, T):
    n, n_t = P.n, P.n_t
    sig = 0.12 * R
    x = -R + np.arange(n) * (2 * R / (n - 1))          # physical node positions
    X, Y = np.meshgrid(x, x)
    g = O.forward(P, np.exp(-(X ** 2 + Y ** 2) / sig ** 2))
    t = np.arange(n_t) * (T / (n_t - 1))                # physical sample times
    ref = np.array([_gauss_physical(sig, c, R, tm) for tm in t])
    return np.linalg.norm(g - ref[None, :]) / (np.linalg.norm(ref) * math.sqrt(P.n_det))


def test_physical_units_centred_gaussian():
    """A at (c, R, T) = (1.5, 0.8, 1.6) against the closed form written in physical units."""
    c, R, T = _PHYS["c"], _PHYS["R"], _PHYS["T"]
    P = O.OraclePlan(64, 128, 128, c=c, R=R, T=T)
    assert _physical_gaussian_error(P, c, R, T) < 5e-4
    # A planted mistake in the normalisation, T' = T R / c instead of c T / R
    # (the same plan with c and R exchanged), is caught.
    bad = O.OraclePlan(64, 128, 128, c=R, R=c, T=T)
    assert _physical_gaussian_error(bad, c, R, T) > 1e-1


def _physical_dot_gap(P, c, R, T, f, g):
    """|<A f, g>_Y - <f, A* g>_X| / |<A f, g>_Y| with the physical quadrature weights."""
    w_x = (2 * R / (P.n - 1)) ** 2                      # dx dy of the node grid on [-R, R]^2
    w_y = (T / (P.n_t - 1)) * (2 * math.pi * R / P.n_det)   # dt times arc length per detector
    lhs = w_y * np.sum(O.forward(P, f) * g)
    rhs = w_x * np.sum(f * O.adjoint(P, g))
    return abs(lhs - rhs) / abs(lhs)


def test_physical_units_dot_product():
    """<A f, g>_Y = <f, A* g>_X (Eq. innerProducts) with weights written here in physical units."""
    c, R, T = _PHYS["c"], _PHYS["R"], _PHYS["T"]
    P = O.OraclePlan(32, 64, 64, c=c, R=R, T=T, support_radius=0.9)
    f = ellipse_phantom(32, 3)
    g = random_sinogram(64, 64, 7)
    assert _physical_dot_gap(P, c, R, T, f, g) <= 1e-12
    # Planted mistakes in the oracle's weights are caught: W_X without R^2, W_Y without R/c.
    for attr, wrong in (("W_X", P.h ** 2), ("W_Y", P.dt * (2 * math.pi * R / P.n_det))):
        bad = O.OraclePlan(32, 64, 64, c=c, R=R, T=T, support_radius=0.9)
        setattr(bad, attr, wrong)
        assert _physical_dot_gap(bad, c, R, T, f, g) > 1e-2


_CS = [(0.3, -0.2, 0.15, 1.0), (-0.25, 0.35, 0.1, 0.7)]


def _fun(x, y):
    return sum(a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / s ** 2) for cx, cy, s, a in _CS)


def _grad(x, y):
    gx = sum(a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / s ** 2) * (-2 * (x - cx) / s ** 2) for cx, cy, s, a in _CS)
    gy = sum(a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / s ** 2) * (-2 * (y - cy) / s ** 2) for cx, cy, s, a in _CS)
    return gx, gy


def test_poisson_formula_second_order():
    """A f against Eq. green_conv for an off-centre smooth phantom; the bilinear error falls 4x per doubling of L."""
    n = 48
    errs = []
    for L in (0.0, 16.0, 32.0):
        P = O.OraclePlan(n, 96, 96, pad_L=L)
        x = -1 + np.arange(n) * P.h
        X, Y = np.meshgrid(x, x)
        g = O.forward(P, _fun(X, Y))
        ds = np.arange(0, 96, 6)
        ms = np.arange(0, 96, 6)
        z = np.stack([np.cos(P.theta[ds]), np.sin(P.theta[ds])], 1)
        ref = O.poisson_truth(_fun, _grad, P.t[ms], z)
        sub = g[np.ix_(ds, ms)]
        errs.append(np.linalg.norm(sub - ref) / np.linalg.norm(ref))
    assert errs[0] < 3e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0
    assert errs[2] < 2e-4


@pytest.mark.parametrize("smooth,n_phi,tol", [(0.05, 0, 1.5e-2), (0.05, 384, 6e-3), (0.0, 384, 1.2e-2)])
def test_kwave_truth(smooth, n_phi, tol):
    """A f against the unaccelerated Fourier method of Eq. kwave on the same frequency grid."""
    P = O.OraclePlan(48, 96, 96, support_radius=0.9, n_phi=n_phi)
    f = ellipse_phantom(48, 0, smooth=smooth)
    g = O.forward(P, f)
    gk = O.kwave_truth(P, f)
    assert np.linalg.norm(g - gk) / np.linalg.norm(gk) < tol


# ------------------------------------------------------------ exact invariants

def test_rotation_by_quarter_turn():
    """Rotating f by +90 degrees cyclically shifts g by n_det/4 detectors (grid and stencils are invariant)."""
    n, nd = 24, 48
    P = O.OraclePlan(n, nd, 40, support_radius=0.9)
    f = ellipse_phantom(n, 5)
    fr = np.empty_like(f)
    for iy in range(n):
        for ix in range(n):
            fr[iy, ix] = f[n - 1 - ix, iy]       # f_rot(x, y) = f(y, -x)
    g = O.forward(P, f)
    gr = O.forward(P, fr)
    assert np.abs(gr - np.roll(g, nd // 4, axis=0)).max() <= 1e-12 * np.abs(g).max()


def test_mirror():
    """y -> -y in f is theta -> -theta in g."""
    n, nd = 24, 48
    P = O.OraclePlan(n, nd, 40, support_radius=0.9)
    f = ellipse_phantom(n, 6)
    g = O.forward(P, f)
    gm = O.forward(P, f[::-1, :])
    assert np.abs(gm - g[(-np.arange(nd)) % nd]).max() <= 1e-12 * np.abs(g).max()


def test_finite_speed_and_linearity():
    """A centred bump of radius ~0.35 is silent at the detectors for t < 0.5; A is linear."""
    n = 48
    P = O.OraclePlan(n, 64, 96, support_radius=0.98)
    x = -1 + np.arange(n) * P.h
    X, Y = np.meshgrid(x, x)
    f = np.exp(-(X ** 2 + Y ** 2) / 0.1 ** 2)
    g = O.forward(P, f)
    early = P.t < 0.5
    assert np.abs(g[:, early]).max() <= 1e-3 * np.abs(g).max()
    f2 = ellipse_phantom(n, 2)
    assert np.allclose(O.forward(P, 2 * f - 3 * f2), 2 * g - 3 * O.forward(P, f2), rtol=0, atol=1e-12)
    assert np.abs(O.forward(P, np.zeros((n, n)))).max() == 0.0


def test_golden_regression():
    """The oracle still reproduces the outputs stored by tests/golden/make_golden.py."""
    import os
    here = os.path.join(os.path.dirname(__file__), "golden")
    gref = np.loadtxt(os.path.join(here, "oracle_n16_forward.txt"))
    fref = np.loadtxt(os.path.join(here, "oracle_n16_adjoint.txt"))
    P = O.OraclePlan(16, 32, 24, support_radius=0.9)
    assert np.abs(O.forward(P, ellipse_phantom(16, 11)) - gref).max() <= 1e-12 * np.abs(gref).max()
    assert np.abs(O.adjoint(P, random_sinogram(32, 24, 12)) - fref).max() <= 1e-12 * np.abs(fref).max()
