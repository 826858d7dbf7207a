"""The plan builder's FP64 tables against the oracle's independent evaluation.

The plan (C++) and the oracle (numpy/scipy) derive grids, Bessel values, the
low-mode quadrature and the bilinear stencils with separate code; these CPU
tests check that they agree before any table is rounded to FP32.
"""
import math

import numpy as np
import pytest
from scipy.special import jv

from oracle import tat_oracle as O


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2510_24687_gb300 as p
    return p


@pytest.mark.parametrize("kw", [
    dict(n=64, n_det=128, n_t=128), dict(n=128, n_det=256, n_t=256), dict(n=256, n_det=512, n_t=512),
    dict(n=512, n_det=1024, n_t=1024), dict(n=1024, n_det=2048, n_t=2048), dict(n=257, n_det=360, n_t=513, T=4.0),
    dict(n=48, n_det=96, n_t=100), dict(n=33, n_det=64, n_t=70), dict(n=64, n_det=128, n_t=128, c=1.5, R=0.8, T=1.6),
    dict(n=64, n_det=128, n_t=128, pad_L=16.0), dict(n=64, n_det=64, n_t=128, n_phi=256),
])
def test_grid_integers_match_oracle(pkg, kw):
    kw = dict(kw)
    c, R, T = kw.pop("c", 1.0), kw.pop("R", 1.0), kw.pop("T", 2.0)
    d = pkg.tat_plan_desc_default(kw["n"], kw["n_det"], kw["n_t"], c, R, T)
    for k in ("n_phi", "pad_L"):
        if k in kw:
            setattr(d, k, kw[k])
    info = pkg.tat_plan_query(d)
    P = O.OraclePlan(kw["n"], kw["n_det"], kw["n_t"], c=c, R=R, T=T, n_phi=kw.get("n_phi", 0),
                     pad_L=kw.get("pad_L", 0.0))
    assert (info["N"], info["M"], info["J"], info["n_phi"]) == (P.N, P.M, P.J, P.n_phi)
    assert abs(info["dlam"] - P.dlam) <= 1e-15 * P.dlam and abs(info["dxi"] - P.dxi) <= 1e-15 * P.dxi


@pytest.mark.parametrize("x", [0.0, 1e-3, 0.5, 3.7, 40.0, 401.3, 802.2, 1606.0])
def test_bessel_table_against_scipy(pkg, x):
    kmax = 1024
    mine = np.array(pkg.tat_debug_bessel(x, kmax))
    ref = jv(np.arange(kmax + 1), x)
    assert np.abs(mine - ref).max() <= 2e-13


def test_low_mode_rule_against_oracle(pkg):
    x, w = pkg.tat_debug_low_mode_rule()
    xo, wo = O.hybrid_rule()
    assert np.abs(np.array(x) - xo).max() <= 1e-13
    assert np.abs(np.array(w) - wo).max() <= 1e-9


def test_stencils_against_oracle(pkg):
    n, nd, nt = 64, 128, 128
    d = pkg.tat_plan_desc_default(n, nd, nt)
    P = O.OraclePlan(n, nd, nt)
    rng = np.random.default_rng(0)
    J = P.J
    rings = list(rng.integers(1, J + 1, 300)) + list(range(J + 1, J + 1 + O.LOW_M)) + [1, J, J]
    lps = list(rng.integers(0, nd // 2, 300)) + [0] * O.LOW_M + [0, 0, nd // 2 - 1]
    i0, k0, a, b = map(np.array, pkg.tat_debug_stencils(d, [int(r) for r in rings], [int(l) for l in lps]))
    radii = np.array([P.lam[r] if r <= J else P.low_lam[r - J - 1] for r in rings])
    phi = 2 * math.pi * (np.array(lps) - nd // 4) / nd
    u = radii * np.cos(phi) / P.dxi
    v = radii * np.sin(phi) / P.dxi
    assert np.abs((i0 + a) - u).max() <= 1e-11 and np.abs((k0 + b) - v).max() <= 1e-11
    assert a.min() >= 0 and a.max() < 1 and b.min() >= 0 and b.max() < 1
    assert i0.min() >= 0 and i0.max() <= P.N // 2 - 2
    assert k0.min() >= -(P.N // 2 - 1) and k0.max() <= P.N // 2 - 2
