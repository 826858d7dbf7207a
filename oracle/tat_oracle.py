"""FP64 CPU oracle of the fast forward operator A and its adjoint A*.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path (``paper_2510_24687_gb300``) and imports nothing from it.

What it computes (Hauptmann, Kunyansky, Poimala, "Fast algorithms enabling
optimization and deep learning for photoacoustic tomography in a circular
detection geometry", arXiv 2510.24687):

* ``forward`` -- Algorithm 1, in the paper's order and notation:
  1. extend f by zero to the square [-L, L]^2 (Section 3.1, L ~ T_new + 2);
  2. 2D FFT -> fhat(xi) on a Cartesian grid, with the unitary convention
     fhat(xi) = (1/2pi) int f(x) exp(-i xi.x) dx (Section 2.1.1);
  3. bilinear interpolation to the polar grid (lambda_j, phi_l);
  4. per ring, Fourier coefficients fhat_k(lambda) in phi (Eq. eq3);
  5. g_k(t) = i^|k| int lambda fhat_k(lambda) J_|k|(lambda) cos(lambda t) dlambda
     (Eq. eq2 / Eq. inverse_cos_tr), a cosine sum on the grid
     lambda_j = j*pi/T_ext, with a quadrature whose nodes cluster at lambda = 0
     for k in {-1, 0, 1} (Section 3.1);
  6. g(t, theta) = sum_k g_k(t) exp(i k theta) (Eq. FourSerForg);
  7. restrict to the detector arc Gamma.
* ``adjoint`` -- the exact transpose of the discrete A under the inner products
  <u, v> = int u v dx and <h, k> = int int h k dz dt (Eq. innerProducts), so
  A* = W_X^{-1} A^T W_Y with W_X = h^2 and W_Y = dt * 2 pi R / n_det.  It runs
  the stages of Algorithm 2 (zero-extend, theta-FFT, cosine transform with the
  (-i)^|k| J_|k| multiplier of Eq. Four_coef_u, phi-series, resampling, 2D
  inverse FFT, restriction to Omega_0), each as the transpose of its forward
  counterpart.
* ``inverse`` -- Algorithm 3, the approximate inverse by the universal
  backprojection formula (Eq. approx_UBP) with the constant C of Eq.
  silly_integral; ``inverse_direct`` evaluates the same formula at the
  Cartesian nodes without the polar grid.
* ``kwave_truth`` -- the unaccelerated Fourier method of Eq. kwave on the same
  Cartesian frequency grid (the paper's own accuracy check, Section 2.1.1).
* ``poisson_truth`` -- the Green's-function form of A, Eq. green_conv.

Readings of passages where the paper is silent or inconsistent are fixed in
``OraclePlan`` (grid rules, cut-off, low-mode rule); each is commented there.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from numpy.polynomial.legendre import leggauss, legval
from scipy.special import bernoulli, jv

TWO_PI = 2.0 * math.pi

# Low-mode quadrature (Section 3.1: for k = -1, 0, 1 the cosine integral is
# evaluated "using a quadrature rule with discretization points clustering
# toward lambda = 0"; the rule itself is not given).  Reading: a hybrid
# Gauss-trapezoidal rule.  The first LOW_A grid nodes j = 0..LOW_A-1 of the
# trapezoid sum are replaced by LOW_M Gauss-Legendre nodes on [0, LOW_A*dlam],
# whose weights make the rule exact (in the Euler-Maclaurin sense) for
# polynomials of degree < LOW_M.
LOW_A = 8
LOW_M = 20


def smooth_ceil(x: float, even: bool = False) -> int:
    """Smallest 2^a 3^b >= x (a >= 1 if ``even``), with a 1e-12 relative slack."""
    target = x * (1.0 - 1e-12)
    best = None
    p2 = 2 if even else 1
    while p2 < 4 * max(target, 1.0) + 4:
        v = p2
        while v < target:
            v *= 3
        if best is None or v < best:
            best = v
        p2 *= 2
    return int(best)


def hybrid_rule(a: int = LOW_A, m: int = LOW_M):
    """Nodes x (in units of dlam, inside (0, a)) and weights w of the low-mode rule.

    The rule  sum_i w_i f(x_i) + sum_{j>=a} f(j)  reproduces int_0^inf f for
    every polynomial f of degree < m in the Euler-Maclaurin sense:
        sum_i w_i q(x_i) = int_0^a q - q(a)/2 + sum_r B_2r/(2r)! q^(2r-1)(a).
    Weights are found in the Legendre basis on [0, a] (well conditioned).
    """
    y, gw = leggauss(m)
    x = a * (y + 1.0) / 2.0
    B = bernoulli(m + 2)
    w = np.zeros(m)
    for p in range(m):
        c = np.zeros(p + 1)
        c[p] = 1.0
        # Evaluated in the Legendre basis on [0, a]: the monomial expansion of
        # P_p(2x/a - 1) cancels catastrophically at x = a for p near m.
        P = np.polynomial.Legendre(c, domain=[0, a])
        prim = P.integ()
        mom = prim(a) - prim(0.0) - 0.5 * P(a)
        d = P.deriv()
        r = 1
        while 2 * r - 1 <= p:
            mom += B[2 * r] / math.factorial(2 * r) * d(a)
            d = d.deriv(2)
            r += 1
        # orthogonal expansion: int_0^a P_p^2 dx = a/(2p+1); GL weights on [0,a] = gw*a/2
        w += gw * (a / 2.0) * ((2 * p + 1) / a) * mom * legval(y, c)
    return x, w


@dataclass
class OraclePlan:
    """Grid sizes of Algorithm 1 derived from the problem statement (Section 2.1).

    Geometry is normalised to R = 1, c = 1 (Section 2.1: "without loss of
    generality"): x' = x/R, t' = c t/R.
    """

    n: int
    n_det: int
    n_t: int
    c: float = 1.0
    R: float = 1.0
    T: float = 2.0
    support_radius: float = 0.98
    arc_begin: float = 0.0
    arc_len: float = TWO_PI
    n_phi: int = 0
    pad_L: float = 0.0
    low_mode: bool = True

    def __post_init__(self):
        n, n_t = self.n, self.n_t
        if n < 2 or n_t < 2 or self.n_det < 4 or self.n_det % 2:
            raise ValueError("invalid sizes")
        if self.c <= 0 or self.R <= 0 or self.T <= 0:
            raise ValueError("c, R, T must be positive")
        self.Tn = self.c * self.T / self.R               # normalised window
        self.h = 2.0 / (n - 1)                           # node-centred grid on [-1,1]
        self.dt = self.Tn / (n_t - 1)                    # t_m = m*dt, m = 0..n_t-1
        # Time extension T_new = max(2T, 6) (Section 3.1) rounded up to M steps.
        self.M = smooth_ceil(max(2.0 * self.Tn, 6.0) / self.dt)
        self.T_ext = self.M * self.dt
        self.dlam = math.pi / self.T_ext                 # DCT-I grid lambda_j = j*dlam
        # Square [-L, L]^2 with L ~ T_new + 2 (Section 3.1); one rule for A and A*.
        self.L = self.pad_L if self.pad_L > 0 else self.T_ext + 2.0
        self.N = smooth_ceil(2.0 * self.L / self.h, even=True)
        if self.N < n:
            self.N = smooth_ceil(float(n), even=True)
        self.dxi = TWO_PI / (self.N * self.h)
        # Radial cut-off: keep every bilinear stencil off the Nyquist row/column.
        lam_c = min(math.pi / self.h - self.dxi, math.pi / self.dt)
        self.lam_c = lam_c
        self.J = min(int(math.ceil(lam_c / self.dlam)) - 1, self.M - 1)
        self.n_phi = self.n_phi or self.n_det
        if self.n_phi % 4 or self.n_phi < self.n_det:
            raise ValueError("n_phi must be a multiple of 4 and >= n_det")
        if self.low_mode and self.J <= LOW_A:
            raise ValueError("radial grid too short for the low-mode rule")
        self.lam = np.arange(self.J + 1) * self.dlam
        self.t = np.arange(n_t) * self.dt
        self.phi = TWO_PI * np.arange(self.n_phi) / self.n_phi
        self.theta = TWO_PI * np.arange(self.n_det) / self.n_det
        # signed angular mode of each phi-DFT bin
        b = np.arange(self.n_phi)
        self.k = np.where(b < self.n_phi // 2, b, b - self.n_phi)
        self.absk = np.abs(self.k)
        # support mask Pi_Omega0: nodes with |x| <= support_radius (ties kept)
        i = np.arange(n)
        s = (2 * i - (n - 1)).astype(np.float64)
        rr = (self.support_radius * (n - 1)) * (self.support_radius * (n - 1))
        self.mask = ((s[:, None] ** 2 + s[None, :] ** 2) <= rr).astype(np.float64)
        # detector arc Gamma: theta_d in [arc_begin, arc_begin + arc_len)
        if self.arc_len >= TWO_PI:
            self.gamma = np.ones(self.n_det)
        else:
            fr = np.arange(self.n_det) / self.n_det - self.arc_begin / TWO_PI
            fr = fr - np.floor(fr)
            self.gamma = (fr < self.arc_len / TWO_PI - 1e-12).astype(np.float64)
        if self.low_mode:
            x, w = hybrid_rule()
            self.low_lam = x * self.dlam
            self.low_w = w
        # inner-product weights of X and Y (physical units)
        self.W_X = (self.h * self.R) ** 2
        self.W_Y = (self.dt * self.R / self.c) * (TWO_PI * self.R / self.n_det)


def _low_bins(P: OraclePlan):
    return [int(np.nonzero(P.k == k)[0][0]) for k in (-1, 0, 1)]


# ----------------------------------------------------------------- forward steps

def spectrum(P: OraclePlan, f: np.ndarray) -> np.ndarray:
    """Steps 1-2: fhat(xi_q) = (h^2/2pi) sum_x f(x) exp(-i xi_q . x) on the N x N grid.

    Returned in FFT order: F[qy mod N, qx mod N], xi_q = q*dxi with q signed.
    """
    n, N = P.n, P.N
    pad = np.zeros((N, N))
    pad[:n, :n] = f * P.mask
    D = np.fft.fft2(pad)
    q = np.fft.fftfreq(N, 1.0 / N)
    ph = np.exp(1j * q * P.dxi)        # exp(-i xi_q x_0) with x_0 = -1
    return (P.h * P.h / TWO_PI) * D * ph[:, None] * ph[None, :]


def _stencil(P: OraclePlan, radii: np.ndarray):
    u = radii[:, None] * np.cos(P.phi)[None, :] / P.dxi
    v = radii[:, None] * np.sin(P.phi)[None, :] / P.dxi
    i0 = np.floor(u)
    k0 = np.floor(v)
    a = u - i0
    b = v - k0
    N = P.N
    i0 = i0.astype(np.int64) % N
    k0 = k0.astype(np.int64) % N
    return i0, (i0 + 1) % N, k0, (k0 + 1) % N, a, b


def polar(P: OraclePlan, F: np.ndarray, radii: np.ndarray) -> np.ndarray:
    """Step 3: bilinear interpolation of the Cartesian grid to (radii x phi_l)."""
    i0, i1, k0, k1, a, b = _stencil(P, radii)
    return ((1 - a) * (1 - b) * F[k0, i0] + a * (1 - b) * F[k0, i1]
            + (1 - a) * b * F[k1, i0] + a * b * F[k1, i1])


def modes(P: OraclePlan, Fp: np.ndarray) -> np.ndarray:
    """Step 4 (Eq. eq3): fhat_k(lambda) = (1/n_phi) sum_l fhat(lambda, phi_l) e^{-ik phi_l}."""
    return np.fft.fft(Fp, axis=1) / P.n_phi


def bessel_table(P: OraclePlan, radii: np.ndarray) -> np.ndarray:
    """J_|k|(lambda) for every radius and phi-DFT bin (stored once per plan)."""
    return jv(P.absk[None, :].astype(np.float64), radii[:, None])


def _cos(P: OraclePlan, radii: np.ndarray) -> np.ndarray:
    return np.cos(radii[:, None] * P.t[None, :])


def cosine_modes(P: OraclePlan, fh: np.ndarray, fh_low: np.ndarray | None) -> np.ndarray:
    """Step 5 (Eq. eq2): g_k(t_m) for every bin k, shape (n_phi, n_t).

    Trapezoid sum over lambda_j = j*dlam (j = 0..J, weight dlam; the j = 0 term
    vanishes with lambda_0 = 0).  For k in {-1, 0, 1} the nodes j < LOW_A are
    replaced by the low-mode nodes (``hybrid_rule``).
    """
    ik = (1j) ** P.absk
    H = ik[None, :] * (P.dlam * P.lam)[:, None] * bessel_table(P, P.lam) * fh
    G = _cos(P, P.lam).T @ H                       # (n_t, n_phi)
    G = G.T.copy()
    if P.low_mode:
        C = _cos(P, P.lam)
        Jl = bessel_table(P, P.low_lam)
        Cl = _cos(P, P.low_lam)
        for b in _low_bins(P):
            hg = H[LOW_A:, b] @ C[LOW_A:, :]
            hl = (ik[b] * P.low_w * P.dlam * P.low_lam * Jl[:, b] * fh_low[:, b]) @ Cl
            G[b] = hg + hl
    return G


def synthesis(P: OraclePlan, G: np.ndarray) -> np.ndarray:
    """Steps 6-7 (Eq. FourSerForg): g(t_m, theta_d) = Re sum_k g_k e^{ik theta_d}, masked to Gamma.

    Returns g[d, m] (detector-major).
    """
    E = np.exp(1j * P.theta[:, None] * P.k[None, :])   # (n_det, n_phi)
    g = (E @ G).real
    return g * P.gamma[:, None]


def forward(P: OraclePlan, f: np.ndarray) -> np.ndarray:
    """g = A f (Algorithm 1).  f: (n, n) with f[iy, ix]; returns g[d, m]."""
    F = spectrum(P, np.asarray(f, dtype=np.float64))
    fh = modes(P, polar(P, F, P.lam))
    fh_low = modes(P, polar(P, F, P.low_lam)) if P.low_mode else None
    return synthesis(P, cosine_modes(P, fh, fh_low))


# ----------------------------------------------------------------- adjoint steps

def adjoint(P: OraclePlan, g: np.ndarray) -> np.ndarray:
    """f = A* g = W_X^{-1} A^T W_Y g (Algorithm 2 stages, each the transpose of Algorithm 1's)."""
    g = np.asarray(g, dtype=np.float64) * P.gamma[:, None] * P.W_Y
    # step 6^T: g'_k(t_m) = sum_d g(t_m, theta_d) e^{-ik theta_d}
    E = np.exp(-1j * P.theta[:, None] * P.k[None, :])
    Gp = (E.T @ g)                                    # (n_phi, n_t)
    # step 5^T: fhat'_k(lambda_j) = (-i)^|k| dlam lambda_j J_|k| sum_m cos(lambda_j t_m) g'_k(t_m)
    ikc = (-1j) ** P.absk
    C = _cos(P, P.lam)
    S = C @ Gp.T                                      # (J+1, n_phi)
    fh = ikc[None, :] * (P.dlam * P.lam)[:, None] * bessel_table(P, P.lam) * S
    if P.low_mode:
        bins = _low_bins(P)
        fh[:LOW_A, bins] = 0.0
        Cl = _cos(P, P.low_lam)
        Jl = bessel_table(P, P.low_lam)
        fh_low = np.zeros((len(P.low_lam), P.n_phi), dtype=np.complex128)
        Sl = Cl @ Gp.T
        for b in bins:
            fh_low[:, b] = ikc[b] * P.low_w * P.dlam * P.low_lam * Jl[:, b] * Sl[:, b]
    # step 4^T: fhat'(lambda, phi_l) = (1/n_phi) sum_k fhat'_k e^{ik phi_l}
    Fp = np.fft.ifft(fh, axis=1)
    Fpl = np.fft.ifft(fh_low, axis=1) if P.low_mode else None
    # step 3^T: bilinear transpose (scatter-add onto the Cartesian grid)
    Fc = np.zeros((P.N, P.N), dtype=np.complex128)
    for radii, vals in ((P.lam, Fp), (P.low_lam, Fpl)) if P.low_mode else ((P.lam, Fp),):
        i0, i1, k0, k1, a, b = _stencil(P, radii)
        np.add.at(Fc, (k0, i0), (1 - a) * (1 - b) * vals)
        np.add.at(Fc, (k0, i1), a * (1 - b) * vals)
        np.add.at(Fc, (k1, i0), (1 - a) * b * vals)
        np.add.at(Fc, (k1, i1), a * b * vals)
    # step 2^T: (h^2/2pi) sum_q F'(q) e^{+i xi_q . x}
    q = np.fft.fftfreq(P.N, 1.0 / P.N)
    ph = np.exp(-1j * q * P.dxi)
    Z = np.fft.ifft2(Fc * ph[:, None] * ph[None, :]) * (P.N * P.N)
    f = (P.h * P.h / TWO_PI) * Z[: P.n, : P.n].real
    # step 1^T and the inner-product weight of X
    return f * P.mask / P.W_X


# ----------------------------------------------------------------- inverse

def inverse_modes(P: OraclePlan, g: np.ndarray) -> np.ndarray:
    """Steps 1-3 of Algorithm 3: vhat_k(lambda_j) on the radial grid, all n_phi mode bins.

    g_k(t_m) = (1/n_det) sum_d g(t_m, theta_d) e^{-ik theta_d} (Eq. FourSerForg, data
    zero off Gamma); the t-integral of Eq. Four_coef_v by the trapezoid rule on
    t_m = m dt (the t = 0 term vanishes), and
        vhat_k(lambda) = -2 (-i)^|k| J'_|k|(lambda) int_0^T g_k(t) sin(lambda t) dt.
    The constant -2 replaces the printed -4 pi: the appendix writes the Fourier
    transform of G without the 1/(2 pi) of the convention that Eq. green_conv
    and Eq. gseries use (with -4 pi, A^{-1} A f would be 2 pi f).
    """
    if P.n_phi != P.n_det:
        raise ValueError("the inverse keeps the data's own modes: n_phi must equal n_det")
    gg = np.asarray(g, dtype=np.float64) * P.gamma[:, None]
    Gk = np.fft.fft(gg, axis=0) / P.n_det                    # (n_phi, n_t), bin order
    w = np.full(P.n_t, P.dt)
    w[-1] *= 0.5
    S = np.sin(np.outer(P.lam, P.t)) @ (w[:, None] * Gk.T)    # (J+1, n_phi)
    ak = P.absk
    dJ = 0.5 * (jv(ak - 1, P.lam[:, None]) - jv(ak + 1, P.lam[:, None]))   # J'_|k|, J_{-1} = -J_1
    return -2.0 * ((-1j) ** ak)[None, :] * dJ * S


def inverse_resample(P: OraclePlan, V: np.ndarray) -> np.ndarray:
    """Step 5: bilinear interpolation in (lambda, phi) of V[j, l] = vhat(lambda_j, phi_l)
    at every Cartesian node xi_q of the N x N grid (FFT order); zero beyond ring J.

    The cut-off is the resampling's only discontinuity; ties u = |xi_q|/dlam = J occur
    exactly on some grids (dxi/dlam rational), so the rule is stated with a margin."""
    q = np.fft.fftfreq(P.N, 1.0 / P.N)
    QX, QY = np.meshgrid(q, q, indexing="xy")
    u = np.hypot(QX, QY) * P.dxi / P.dlam
    # Closed cut-off: nodes up to ring J (within 1e-6 of a cell, so that exact
    # rational ties such as u = J are inside whatever the rounding) take the
    # interpolated value; beyond it vhat = 0.
    inside = u <= P.J + 1e-6
    j0 = np.minimum(np.floor(u).astype(np.int64), P.J - 1)
    a = np.minimum(u - j0, 1.0)
    j0 = np.where(inside, j0, 0)
    s = (np.arctan2(QY, QX) / TWO_PI * P.n_phi) % P.n_phi
    l0 = np.floor(s).astype(np.int64)
    b = s - l0
    l0 %= P.n_phi
    l1 = (l0 + 1) % P.n_phi
    out = ((1 - a) * ((1 - b) * V[j0, l0] + b * V[j0, l1]) + a * ((1 - b) * V[j0 + 1, l0] + b * V[j0 + 1, l1]))
    return np.where(inside, out, 0.0)


def _annulus(P: OraclePlan) -> np.ndarray:
    """Nodes of Omega \\ Omega_0: inside the disk |x| <= R, outside the support mask."""
    i = np.arange(P.n)
    s = (2 * i - (P.n - 1)).astype(np.float64)
    inside = (s[:, None] ** 2 + s[None, :] ** 2) <= float(P.n - 1) ** 2
    return inside & (P.mask == 0)


def inverse(P: OraclePlan, g: np.ndarray, with_constant: bool = True) -> np.ndarray:
    """f ~ A^{-1} g (Algorithm 3): universal backprojection (Eq. approx_UBP) on the grids of A*.

    Steps: detector DFT and sine transform (inverse_modes), angular series
    vhat(lambda_j, phi_l) = sum_k e^{ik phi_l} vhat_k (step 4), bilinear resampling to
    the Cartesian grid (step 5), the 2D inverse transform
    v(x) = (dxi^2 / 2 pi) sum_q vhat(xi_q) e^{i xi_q . x} on the image nodes (step 6),
    C = -mean of v over Omega \\ Omega_0 (Eq. silly_integral, step 7) and
    Pi_Omega0 (v + C) (step 8).
    """
    V = np.fft.ifft(inverse_modes(P, g), axis=1) * P.n_phi
    Vc = inverse_resample(P, V)
    q = np.fft.fftfreq(P.N, 1.0 / P.N)
    ph = np.exp(-1j * q * P.dxi)                      # e^{i xi_q x_0}, x_0 = -1
    Z = np.fft.ifft2(Vc * ph[:, None] * ph[None, :]) * (P.N * P.N)
    v = (P.dxi * P.dxi / TWO_PI) * Z[: P.n, : P.n].real
    ann = _annulus(P)
    C = -v[ann].mean() if (with_constant and ann.any()) else 0.0
    return (v + C) * P.mask


def inverse_direct(P: OraclePlan, g: np.ndarray) -> np.ndarray:
    """Algorithm 3 without the polar grid: vhat evaluated at every Cartesian node by the
    mode sum of Eq. Four_ser_v with the exact J'_|k|(|xi|) and sin(|xi| t) (no
    interpolation), then steps 6-8.  O(N^2 n_phi n_t): tiny grids only."""
    gg = np.asarray(g, dtype=np.float64) * P.gamma[:, None]
    Gk = np.fft.fft(gg, axis=0) / P.n_det
    w = np.full(P.n_t, P.dt)
    w[-1] *= 0.5
    q = np.fft.fftfreq(P.N, 1.0 / P.N)
    QX, QY = np.meshgrid(q, q, indexing="xy")
    lam = (np.hypot(QX, QY) * P.dxi).ravel()
    phi = np.arctan2(QY, QX).ravel()
    keep = lam / P.dlam <= P.J + 1e-6
    Vc = np.zeros(lam.size, dtype=np.complex128)
    L, F = lam[keep], phi[keep]
    S = np.sin(np.outer(L, P.t)) @ (w[:, None] * Gk.T)         # (nodes, n_phi)
    ak = P.absk
    dJ = 0.5 * (jv(ak[None, :] - 1, L[:, None]) - jv(ak[None, :] + 1, L[:, None]))
    E = np.exp(1j * F[:, None] * P.k[None, :])
    Vc[keep] = (-2.0 * ((-1j) ** ak)[None, :] * dJ * S * E).sum(axis=1)
    Vc = Vc.reshape(P.N, P.N)
    ph = np.exp(-1j * q * P.dxi)
    Z = np.fft.ifft2(Vc * ph[:, None] * ph[None, :]) * (P.N * P.N)
    v = (P.dxi * P.dxi / TWO_PI) * Z[: P.n, : P.n].real
    ann = _annulus(P)
    C = -v[ann].mean() if ann.any() else 0.0
    return (v + C) * P.mask


# ----------------------------------------------------------------- slow truths

def kwave_truth(P: OraclePlan, f: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """Eq. kwave without acceleration: g(t_m, z_d) = (dxi^2/2pi) sum_{|xi|<=lam_J} fhat(xi) cos(|xi| t_m) e^{i xi.z_d}.

    The same Cartesian frequency grid as ``spectrum``; no interpolation, no
    angular or cosine transform.  O(N^2 n_det n_t): tiny grids only.
    """
    F = spectrum(P, f)
    q = np.fft.fftfreq(P.N, 1.0 / P.N) * P.dxi
    QX, QY = np.meshgrid(q, q, indexing="xy")
    lam = np.hypot(QX, QY)
    sel = lam <= P.lam[-1] + 1e-12
    xs, ys, ls, Fs = QX[sel], QY[sel], lam[sel], F[sel]
    zx, zy = np.cos(P.theta), np.sin(P.theta)
    g = np.zeros((P.n_det, P.n_t))
    for s in range(0, len(ls), chunk):
        e = np.exp(1j * (np.outer(zx, xs[s:s + chunk]) + np.outer(zy, ys[s:s + chunk])))
        c = np.cos(np.outer(ls[s:s + chunk], P.t))
        g += ((e * Fs[None, s:s + chunk]) @ c).real
    return g * (P.dxi ** 2 / TWO_PI) * P.gamma[:, None]


def poisson_truth(fun, grad, t: np.ndarray, z: np.ndarray, n_beta: int = 64, n_alpha: int = 256) -> np.ndarray:
    """Eq. green_conv evaluated directly for a smooth f given analytically.

    g(t, z) = d/dt int f(x) G(t, x - z) dx with G = 1/(2pi sqrt(t^2-|x|^2)).
    With y = t sin(beta) e_alpha the time derivative becomes
    g = (1/2pi) int_0^{pi/2} int_0^{2pi} sin(beta) [f + t sin(beta) e_alpha . grad f](z + t sin(beta) e_alpha) dalpha dbeta,
    evaluated by Gauss-Legendre in beta and the trapezoid rule in alpha.
    ``z``: (nz, 2) points; returns (nz, len(t)).
    """
    yb, wb = leggauss(n_beta)
    beta = (yb + 1.0) * math.pi / 4.0
    wb = wb * math.pi / 4.0
    alpha = TWO_PI * np.arange(n_alpha) / n_alpha
    ea = np.stack([np.cos(alpha), np.sin(alpha)], axis=-1)
    out = np.zeros((len(z), len(t)))
    for iz, zz in enumerate(z):
        for it, tt in enumerate(t):
            r = tt * np.sin(beta)                                  # (nb,)
            pts = zz[None, None, :] + r[:, None, None] * ea[None, :, :]
            fv = fun(pts[..., 0], pts[..., 1])
            gx, gy = grad(pts[..., 0], pts[..., 1])
            dirder = gx * ea[None, :, 0] + gy * ea[None, :, 1]
            integ = np.sin(beta)[:, None] * (fv + r[:, None] * dirder)
            # (1/2pi) * int dalpha  ==  mean over the uniform alpha nodes
            out[iz, it] = wb @ integ.mean(axis=1)
    return out
