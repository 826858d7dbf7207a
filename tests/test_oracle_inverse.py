"""Pins of the FP64 oracle of the approximate inverse A^{-1} (Algorithm 3).

The inverse is pinned against what the mathematics fixes, not against itself:
the universal backprojection formula is a left inverse of A for complete data
and T -> infinity (Eq. inverse), so A^{-1} A f must return a smooth f up to a
small error that falls as T grows (the paper reports 0.22 % relative L2 for its
phantom with T = 4, Section 4.3); the same formula evaluated at the Cartesian
nodes without the polar grid must agree with the fast path up to the bilinear
interpolation error; and exact symmetries of the grids (quarter turn, mirror)
must hold to rounding.
"""
import numpy as np

from oracle import tat_oracle as O


def bump(P, cx=0.2, cy=-0.1, w=0.15):
    x = -1 + P.h * np.arange(P.n)
    X, Y = np.meshgrid(x, x)
    return np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * w * w)) * P.mask


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_left_inverse_on_complete_data():
    """A^{-1} A f = f for a smooth off-centre bump, full circle, T = 4: 0.17 % (paper: 0.22 % for its
    phantom); the finite-time error shrinks at T = 6; a wrong sign, factor or angle convention fails."""
    P4 = O.OraclePlan(64, 128, 128, T=4.0, support_radius=0.98)
    f = bump(P4)
    e4 = rel(O.inverse(P4, O.forward(P4, f)), f)
    P6 = O.OraclePlan(64, 128, 128, T=6.0, support_radius=0.98)
    e6 = rel(O.inverse(P6, O.forward(P6, f)), f)
    assert e4 < 3e-3
    assert e6 < 0.7 * e4


def test_constant_reduces_finite_time_error():
    """The constant C of Eq. silly_integral lowers the error of the truncated-time reconstruction."""
    P = O.OraclePlan(64, 128, 128, T=4.0, support_radius=0.98)
    f = bump(P)
    g = O.forward(P, f)
    assert rel(O.inverse(P, g), f) < 0.8 * rel(O.inverse(P, g, with_constant=False), f)


def test_direct_evaluation_agrees_up_to_interpolation():
    """Without the polar grid (exact vhat at every Cartesian node) the formula recovers f to 6e-4;
    the fast path differs from it by the bilinear interpolation error, which falls with the grid."""
    d = {}
    for n in (16, 32):
        P = O.OraclePlan(n, 2 * n, 2 * n, T=4.0, support_radius=0.98)
        f = bump(P)
        g = O.forward(P, f)
        fd = O.inverse_direct(P, g)
        d[n] = rel(O.inverse(P, g), fd)
        if n == 32:
            assert rel(fd, f) < 1e-3
    assert d[32] < 4e-3 and d[32] < 0.5 * d[16]


def test_quarter_turn_and_mirror():
    """Rolling the data by n_det/4 detectors rotates the reconstruction by +90 degrees; reversing theta
    mirrors it in y (exact symmetries of the grids and of the resampling)."""
    n, nd = 24, 48
    P = O.OraclePlan(n, nd, 40, T=2.0, support_radius=0.9)
    rng = np.random.default_rng(3)
    g = rng.standard_normal((nd, 40))
    f = O.inverse(P, g)
    fr = O.inverse(P, np.roll(g, nd // 4, axis=0))
    rot = np.empty_like(f)
    for iy in range(n):
        for ix in range(n):
            rot[iy, ix] = f[n - 1 - ix, iy]          # f_rot(x, y) = f(y, -x)
    assert np.abs(fr - rot).max() <= 1e-12 * np.abs(f).max()
    fm = O.inverse(P, g[(-np.arange(nd)) % nd])
    assert np.abs(fm - f[::-1, :]).max() <= 1e-12 * np.abs(f).max()
