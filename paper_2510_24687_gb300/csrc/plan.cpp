// Host plan builder: derives the grids of Algorithm 1 / Algorithm 2 and
// computes every table in FP64 before rounding it to FP32 for the device.
//
// Grid rules (Section 3.1), one set shared by A and A*:
//   h = 2/(n-1) (node-centred image grid on [-1,1]^2 after scaling by R),
//   dt = T'/(n_t-1) with T' = cT/R,
//   T_new = M*dt, M = smallest 2^a3^b >= max(2T', 6)/dt  (time extension),
//   L = T_new + 2 (padded square [-L, L]^2), N = smallest even 2^a3^b >= 2L/h,
//   dxi = 2 pi/(N h), dlam = pi/T_new, lambda_j = j*dlam for j = 0..J with
//   J*dlam < min(pi/h - dxi, pi/dt) so that no bilinear stencil touches the
//   unpaired Nyquist row or column of the N x N spectrum.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>
#include <vector>

#include "plan.hpp"

#define TAT_TRY(x)               \
  do {                           \
    tat_status s_ = (x);         \
    if (s_ != TAT_OK) return s_; \
  } while (0)

namespace tat {

namespace {
constexpr double kPi = 3.14159265358979323846264338327950288;

using cd = std::complex<double>;

// In-place iterative radix-2 FFT (forward sign), length a power of two.
void fft_pow2(std::vector<cd>& a, const std::vector<cd>& tw) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const size_t step = n / len;
    for (size_t i = 0; i < n; i += len) {
      for (size_t k = 0; k < len / 2; ++k) {
        const cd w = tw[k * step];
        const cd u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
    }
  }
}

template <class F>
void parallel_for(int count, F&& fn) {
  unsigned hw = std::thread::hardware_concurrency();
  int nth = (int)std::max(1u, std::min(hw == 0 ? 1u : hw, 32u));
  nth = std::min(nth, std::max(1, count / 8));
  if (nth <= 1) {
    for (int i = 0; i < count; ++i) fn(i);
    return;
  }
  std::vector<std::thread> th;
  for (int t = 0; t < nth; ++t)
    th.emplace_back([&, t]() {
      for (int i = t; i < count; i += nth) fn(i);
    });
  for (auto& x : th) x.join();
}

// Radix schedule: radix-3 passes, radix-16 passes, then the remainder of
// log2 mod 4 as 8*4 (one 16 fewer), 4 or 8 (or one 2 for a length-2 factor);
// the device code uses the same rule.
int fft_schedule(int L, int* radix, int order = 0) {
  int r = L, np = 0;
  while (r % 3 == 0) { radix[np++] = 3; r /= 3; }
  int k = 0;
  while ((1 << k) < r) ++k;
  if ((1 << k) != r) return -1;
  const int n16full = k / 4, rem = k % 4;
  const int n16 = (rem == 1 && n16full >= 1) ? n16full - 1 : n16full;
  for (int i = 0; i < n16; ++i) radix[np++] = 16;
  if (rem == 1) {
    if (n16full >= 1) { radix[np++] = 8; radix[np++] = 4; }
    else radix[np++] = 2;
  } else if (rem == 2) {
    radix[np++] = 4;
  } else if (rem == 3) {
    radix[np++] = 8;
  }
  if (order == 1) std::reverse(radix, radix + np);  // the same passes, tail radix first
  return np;
}

// Smallest multiple of 32 threads for which every pass holds <= 16 values per thread.
int fft_threads(const FftDev& f) {
  for (int nt = 32; nt <= 1024; nt += 32) {
    bool ok = true;
    for (int s = 0; s < f.npass; ++s) {
      const int R = f.radix[s];
      const int per = (f.L / R + nt - 1) / nt;
      if (per * R > 16) ok = false;
    }
    if (ok) return nt;
  }
  return -1;
}

}  // namespace

long long smooth_ceil(double x, bool even) {
  const double target = x * (1.0 - 1e-12);
  long long best = -1;
  for (long long p2 = even ? 2 : 1; p2 < 4 * std::max(target, 1.0) + 4; p2 *= 2) {
    long long v = p2;
    while ((double)v < target) v *= 3;
    if (best < 0 || v < best) best = v;
  }
  return best;
}

// cos and sin of 2 pi num/den, reduced to the first octant in exact integer
// arithmetic so that multiples of pi/2 are exact and mirrored angles give
// exactly mirrored values.
void cos_sin_2pi(long long num, long long den, double* c, double* s) {
  long long r = num % den;
  if (r < 0) r += den;
  const long long q = (4 * r) / den;        // quadrant
  const long long rem = 4 * r - q * den;    // angle in the quadrant = (pi/2) rem/den
  double c0, s0;
  if (2 * rem <= den) {
    const double a = (kPi / 2) * ((double)rem / (double)den);
    c0 = std::cos(a);
    s0 = std::sin(a);
  } else {
    const double a = (kPi / 2) * ((double)(den - rem) / (double)den);
    c0 = std::sin(a);
    s0 = std::cos(a);
  }
  if (rem == 0) { c0 = 1.0; s0 = 0.0; }
  switch (q) {
    case 0: *c = c0; *s = s0; break;
    case 1: *c = -s0; *s = c0; break;
    case 2: *c = -c0; *s = -s0; break;
    default: *c = s0; *s = -c0; break;
  }
}

// J_k(x) for k = 0..kmax from the Jacobi-Anger expansion (Eq. Anger):
// e^{i x sin(tau)} = sum_k J_k(x) e^{i k tau}, so the P-point DFT of the
// samples e^{i x sin(2 pi p/P)} returns J_k(x) plus aliases J_{k +- P}(x),
// which are below 1e-17 once P - kmax exceeds x by a margin.
void bessel_orders(double x, int kmax, double* out) {
  const double need = x + kmax + 64 + 16 * std::cbrt(std::max(x, 1.0));
  size_t P = 64;
  while ((double)P < need || (int)P < 2 * kmax + 2) P <<= 1;
  std::vector<cd> tw(P / 2), a(P);
  for (size_t k = 0; k < P / 2; ++k) {
    double c, s;
    cos_sin_2pi(-(long long)k, (long long)P, &c, &s);
    tw[k] = cd(c, s);
  }
  for (size_t p = 0; p < P; ++p) {
    double c, s;
    cos_sin_2pi((long long)p, (long long)P, &c, &s);
    const double ph = x * s;
    a[p] = cd(std::cos(ph), std::sin(ph));
  }
  fft_pow2(a, tw);
  for (int k = 0; k <= kmax; ++k) out[k] = a[k].real() / (double)P;
}

// Nodes (in units of dlam) and weights of the low-mode quadrature: kLowM
// Gauss-Legendre nodes on [0, a], a = kLowA, with weights chosen so that
//   sum_i w_i q(x_i) + sum_{j >= a} q(j)
// equals int_0^inf q in the Euler-Maclaurin sense for every polynomial q of
// degree < kLowM, i.e.
//   sum_i w_i q(x_i) = int_0^a q - q(a)/2 + sum_r B_2r/(2r)! q^(2r-1)(a).
// The weights are expanded in Legendre polynomials on [0, a].
void low_mode_rule(double* nodes, double* weights) {
  const int m = kLowM;
  const double a = (double)kLowA;
  // Gauss-Legendre on [-1, 1] by Newton iteration on P_m.
  std::vector<double> y(m), gw(m);
  auto legendre = [m](double z, double* pm, double* dpm) {
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= m; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    *pm = p1;
    *dpm = m * (z * p1 - p0) / (z * z - 1.0);
  };
  for (int i = 0; i < m; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (m + 0.5)), pm, dpm;
    for (int it = 0; it < 100; ++it) {
      legendre(z, &pm, &dpm);
      const double dz = pm / dpm;
      z -= dz;
      if (std::fabs(dz) <= 1e-15) break;
    }
    legendre(z, &pm, &dpm);
    y[i] = z;
    gw[i] = 2.0 / ((1.0 - z * z) * dpm * dpm);
  }
  // Bernoulli numbers B_0..B_m by sum_{k<=j} C(j+1,k) B_k = 0.
  std::vector<double> B(m + 2, 0.0);
  B[0] = 1.0;
  for (int j = 1; j <= m; ++j) {
    double acc = 0.0, binom = 1.0;  // C(j+1, 0)
    for (int k = 0; k < j; ++k) {
      acc += binom * B[k];
      binom = binom * (double)(j + 1 - k) / (double)(k + 1);
    }
    B[j] = -acc / (double)(j + 1);
  }
  auto fact = [](int k) { double f = 1.0; for (int i = 2; i <= k; ++i) f *= i; return f; };
  // Regularised moments of P_p(2x/a - 1).  Derivative at x = a:
  // (2/a)^s P_p^(s)(1) with P_p^(s)(1) = (p+s)!/(2^s s! (p-s)!).
  std::vector<double> mu(m);
  for (int p = 0; p < m; ++p) {
    double v = (p == 0 ? a : 0.0) - 0.5;
    for (int r = 1; 2 * r - 1 <= p; ++r) {
      const int s = 2 * r - 1;
      const double dP = fact(p + s) / (std::pow(2.0, s) * fact(s) * fact(p - s));
      v += B[2 * r] / fact(2 * r) * std::pow(2.0 / a, s) * dP;
    }
    mu[p] = v;
  }
  for (int i = 0; i < m; ++i) {
    double acc = 0.0, p0 = 1.0, p1 = y[i];
    for (int p = 0; p < m; ++p) {
      double Pp;
      if (p == 0) Pp = 1.0;
      else if (p == 1) Pp = y[i];
      else {
        const double p2 = ((2.0 * p - 1.0) * y[i] * p1 - (p - 1.0) * p0) / p;
        p0 = p1;
        p1 = p2;
        Pp = p2;
      }
      acc += 0.5 * (2 * p + 1) * mu[p] * Pp;
    }
    // store in increasing node order (Newton produced decreasing y)
    nodes[m - 1 - i] = a * (y[i] + 1.0) / 2.0;
    weights[m - 1 - i] = gw[i] * acc;
  }
}

namespace {

template <class T>
tat_status upload(tat_plan_s* P, const std::vector<T>& h, const T** out) {
  void* d = nullptr;
  const size_t bytes = std::max<size_t>(h.size() * sizeof(T), 16);
  if (cudaMalloc(&d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return TAT_ERR_OOM;
  }
  P->allocations.push_back(d);
  if (!h.empty() && cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return TAT_ERR_CUDA;
  *out = static_cast<const T*>(d);
  return TAT_OK;
}

tat_status make_fft(tat_plan_s* P, int L, FftDev* f, int* nthreads, int order = 0) {
  f->L = L;
  f->npass = fft_schedule(L, f->radix, order);
  if (f->npass < 0 || f->npass > kMaxPass) return TAT_ERR_UNSUPPORTED;
  std::vector<float2> tw(L);
  for (int k = 0; k < L; ++k) {
    double c, s;
    cos_sin_2pi(k, L, &c, &s);
    tw[k] = make_float2((float)c, (float)-s);
  }
  *nthreads = fft_threads(*f);
  if (*nthreads < 0) return TAT_ERR_UNSUPPORTED;
  TAT_TRY(upload(P, tw, &f->tw));
  // per-pass base-power tables (see FftDev)
  std::vector<float2> pt;
  long long Ns = 1;
  for (int s = 0; s < f->npass; ++s) {
    const int R = f->radix[s];
    f->ptw_off[s] = (int)pt.size();
    if (s > 0) {
      const long long den = Ns * R;
      auto push = [&](long long k, int p) {
        double c, sn;
        cos_sin_2pi(-k * p, den, &c, &sn);
        pt.push_back(make_float2((float)c, (float)sn));
      };
      const int pw[4] = {1, 2, 4, 8};
      if (Ns <= 16 || Ns % 16) {
        for (int pi = 0; pi < 4; ++pi)
          for (long long k = 0; k < Ns; ++k) push(k, pw[pi]);
      } else {
        for (int pi = 0; pi < 4; ++pi)
          for (long long a = 0; a < Ns / 16; ++a) push(16 * a, pw[pi]);
        for (int pi = 0; pi < 4; ++pi)
          for (long long b = 0; b < 16; ++b) push(b, pw[pi]);
      }
    }
    Ns *= R;
  }
  f->ptw_len = (int)pt.size();
  TAT_TRY(upload(P, pt, &f->ptw));
  // Four-step twiddles for L = RA*256 (RA = 2, 4, 8, 16, 32):
  // w_L^(16 a p), w_L^(b p), w_256^(m p) for a, b, m < 16 and p = 1, 2, 4, 8.
  std::vector<float2> ft(192, make_float2(1.f, 0.f));
  if (L % 256 == 0 && (L / 256 == 2 || L / 256 == 4 || L / 256 == 8 || L / 256 == 16 || L / 256 == 32)) {
    const int pw[4] = {1, 2, 4, 8};
    for (int pi = 0; pi < 4; ++pi)
      for (int i = 0; i < 16; ++i) {
        double c, sn;
        cos_sin_2pi(-(long long)16 * i * pw[pi], L, &c, &sn);
        ft[pi * 16 + i] = make_float2((float)c, (float)sn);
        cos_sin_2pi(-(long long)i * pw[pi], L, &c, &sn);
        ft[64 + pi * 16 + i] = make_float2((float)c, (float)sn);
        cos_sin_2pi(-(long long)i * pw[pi], 256, &c, &sn);
        ft[128 + pi * 16 + i] = make_float2((float)c, (float)sn);
      }
  }
  return upload(P, ft, &f->fstw);
}

}  // namespace

// Grid integers of a problem (host only, no CUDA).
tat_status derive_grids(const tat_plan_desc& D, Grids* G) {
  if (D.n < 8 || D.n_det < 8 || (D.n_det % 2) || D.n_t < 8) return TAT_ERR_INVALID_ARG;
  if (!(D.c > 0) || !(D.R > 0) || !(D.T > 0) || !(D.support_radius > 0) || !(D.arc_len > 0))
    return TAT_ERR_INVALID_ARG;
  if (D.n_phi < 0 || D.pad_L < 0) return TAT_ERR_INVALID_ARG;
  const int n = D.n, n_t = D.n_t;
  G->Tn = D.c * D.T / D.R;
  G->h = 2.0 / (n - 1);
  G->dt = G->Tn / (n_t - 1);
  G->M = smooth_ceil(std::max(2.0 * G->Tn, 6.0) / G->dt, false);
  G->T_ext = (double)G->M * G->dt;
  G->dlam = kPi / G->T_ext;
  const double L = D.pad_L > 0 ? D.pad_L : G->T_ext + 2.0;
  G->N = smooth_ceil(2.0 * L / G->h, true);
  if (G->N < n) G->N = smooth_ceil((double)n, true);
  G->dxi = 2.0 * kPi / ((double)G->N * G->h);
  G->lam_c = std::min(kPi / G->h - G->dxi, kPi / G->dt);
  G->J = std::min((long long)std::ceil(G->lam_c / G->dlam) - 1, G->M - 1);
  G->n_phi = D.n_phi ? D.n_phi : D.n_det;
  if (G->n_phi % 4 || G->n_phi < D.n_det) return TAT_ERR_INVALID_ARG;
  if (G->N > 16384 || 2 * G->M > 16384 || G->n_phi > 16384 || G->J < 2) return TAT_ERR_UNSUPPORTED;
  G->low_on = D.low_mode_quadrature != 0;
  if (G->low_on && G->J <= kLowA) return TAT_ERR_UNSUPPORTED;
  return TAT_OK;
}

void fill_info(const Grids& G, tat_plan_info* I) {
  I->N = (int)G.N; I->M = (int)G.M; I->J = (int)G.J; I->n_phi = G.n_phi; I->K = G.n_phi / 2;
  I->n_low = G.low_on ? kLowM : 0;
  I->n_points = (int)((G.J + I->n_low) * (G.n_phi / 2));
  I->h = G.h; I->dt = G.dt; I->dlam = G.dlam; I->dxi = G.dxi; I->lam_c = G.lam_c;
}

tat_status build_plan(const tat_plan_desc& D, tat_plan_s* P) {
  Grids G;
  TAT_TRY(derive_grids(D, &G));
  P->desc = D;
  DevPlan& d = P->d;
  const int n = D.n, n_t = D.n_t, n_det = D.n_det;
  const double h = G.h, dt = G.dt, dlam = G.dlam, dxi = G.dxi;
  const long long N = G.N, M = G.M, J = G.J;
  const int n_phi = G.n_phi;
  const bool low_on = G.low_on;
  fill_info(G, &P->info);

  d.n = n; d.n_det = n_det; d.n_t = n_t;
  d.N = (int)N; d.M = (int)M; d.J = (int)J; d.n_phi = n_phi; d.K = n_phi / 2; d.nh = n_phi / 2;
  d.n_low = low_on ? kLowM : 0;
  d.n_rings = d.J + 1 + d.n_low;
  d.ncol = d.N / 2;
  d.low_on = low_on ? 1 : 0;
  d.h2_2pi = (float)(h * h / (2.0 * kPi));
  d.adj_scale = (float)(dt / (D.c * n_det));


  // FFT lengths: N (rows/columns), n_phi (rings), 2M (cosine transform), n_det (detectors).
  TAT_TRY(make_fft(P, d.N, &d.fN, &P->cfg.nt_N));
  TAT_TRY(make_fft(P, n_phi, &d.fphi, &P->cfg.nt_phi));
  // the cosine/sine transforms' FFT in both pass orders (the autotuner picks one per plan)
  TAT_TRY(make_fft(P, 2 * d.M, &P->f2M_v[0], &P->nt_2M_v[0], 0));
  TAT_TRY(make_fft(P, 2 * d.M, &P->f2M_v[1], &P->nt_2M_v[1], 1));
  d.f2M = P->f2M_v[0];
  P->cfg.nt_2M = P->nt_2M_v[0];
  P->cfg.order_2M = 0;
  TAT_TRY(make_fft(P, n_det, &d.fdet, &P->cfg.nt_det));

  // Phase e^{-i xi_q x_0} = e^{i q dxi} (x_0 = -1) of every FFT bin, q signed:
  // q dxi = pi q (n-1)/N, reduced exactly.
  {
    std::vector<float2> ph(d.N);
    for (int q = 0; q < d.N; ++q) {
      const long long qs = q < d.N / 2 ? q : (long long)q - d.N;
      double c, s;
      cos_sin_2pi(qs * (n - 1), 2LL * d.N, &c, &s);
      ph[q] = make_float2((float)c, (float)s);
    }
    TAT_TRY(upload(P, ph, &d.phase));
    // Two-level form for the column kernels' shared memory: with q unsigned,
    // e^{2 pi i q (n-1)/(2N)} = hi[q >> 6] lo[q & 63]; the signed bins q >= N/2 differ
    // by e^{-i pi (n-1)} = (-1)^(n-1).
    d.ph_lo = (d.N + 63) / 64;
    d.ph_flip = (n - 1) & 1;
    std::vector<float2> ph2(d.ph_lo + 64);
    for (int a = 0; a < d.ph_lo; ++a) {
      double c, s;
      cos_sin_2pi(64LL * a * (n - 1), 2LL * d.N, &c, &s);
      ph2[a] = make_float2((float)c, (float)s);
    }
    for (int b = 0; b < 64; ++b) {
      double c, s;
      cos_sin_2pi((long long)b * (n - 1), 2LL * d.N, &c, &s);
      ph2[d.ph_lo + b] = make_float2((float)c, (float)s);
    }
    TAT_TRY(upload(P, ph2, &d.phase2));
  }
  // Support disk Pi_Omega0: node kept iff (2ix-(n-1))^2 + (2iy-(n-1))^2 <= (r (n-1))^2.
  {
    const double rr = (D.support_radius * (n - 1)) * (D.support_radius * (n - 1));
    std::vector<int2> rr_rows(n);
    for (int iy = 0; iy < n; ++iy) {
      int lo = n, hi = 0;
      const double sy = 2.0 * iy - (n - 1);
      for (int ix = 0; ix < n; ++ix) {
        const double sx = 2.0 * ix - (n - 1);
        if (sx * sx + sy * sy <= rr) { lo = std::min(lo, ix); hi = ix + 1; }
      }
      if (hi == 0) lo = 0;
      rr_rows[iy] = make_int2(lo, hi);
    }
    TAT_TRY(upload(P, rr_rows, &d.rowrange));
    // The disk Omega inside the detector circle (|x| <= R: (2ix-(n-1))^2 + (2iy-(n-1))^2 <= (n-1)^2)
    // and the node count of Omega \ Omega0, over which the inverse's constant C is fixed.
    const double ro = (double)(n - 1) * (double)(n - 1);
    std::vector<int2> out_rows(n);
    long long ring_nodes = 0;
    for (int iy = 0; iy < n; ++iy) {
      int lo = n, hi = 0;
      const double sy = 2.0 * iy - (n - 1);
      for (int ix = 0; ix < n; ++ix) {
        const double sx = 2.0 * ix - (n - 1);
        if (sx * sx + sy * sy <= ro) {
          lo = std::min(lo, ix);
          hi = ix + 1;
          if (!(ix >= rr_rows[iy].x && ix < rr_rows[iy].y)) ++ring_nodes;
        }
      }
      if (hi == 0) lo = 0;
      out_rows[iy] = make_int2(lo, hi);
    }
    TAT_TRY(upload(P, out_rows, &d.outrange));
    d.inv_count = (float)ring_nodes;
  }
  // Detector arc Gamma.
  {
    std::vector<float> gam(n_det, 1.0f);
    if (D.arc_len < 2.0 * kPi) {
      for (int dd = 0; dd < n_det; ++dd) {
        double fr = (double)dd / (double)n_det - D.arc_begin / (2.0 * kPi);
        fr = fr - std::floor(fr);
        gam[dd] = fr < D.arc_len / (2.0 * kPi) - 1e-12 ? 1.0f : 0.0f;
      }
    }
    TAT_TRY(upload(P, gam, &d.gamma));
  }
  // Radii of every ring: j*dlam for j = 0..J, then the low-mode nodes.
  std::vector<double> lam(d.n_rings);
  std::vector<double> lw(kLowM, 0.0), lx(kLowM, 0.0);
  for (int j = 0; j <= d.J; ++j) lam[j] = (double)j * dlam;
  if (low_on) {
    low_mode_rule(lx.data(), lw.data());
    for (int q = 0; q < kLowM; ++q) lam[d.J + 1 + q] = lx[q] * dlam;
  }
  // Bessel table J_k(lambda_r) for k = 0..K+1 (Section 3.1: precomputed once per plan;
  // order K+1 enters J'_K of the inverse).
  const int KS = d.K + 2;
  std::vector<double> Jt((size_t)d.n_rings * KS);
  parallel_for(d.n_rings, [&](int r) { bessel_orders(lam[r], d.K + 1, &Jt[(size_t)r * KS]); });
  {
    std::vector<float> Bt((size_t)(d.K + 1) * (d.J + 1));
    for (int k = 0; k <= d.K; ++k)
      for (int j = 0; j <= d.J; ++j)
        Bt[(size_t)k * (d.J + 1) + j] = (float)(dlam * lam[j] * Jt[(size_t)j * KS + k] / n_phi);
    TAT_TRY(upload(P, Bt, &d.Bt));
    // Inverse (Eq. Four_coef_v): J'_0 = -J_1, J'_k = (J_{k-1} - J_{k+1}) / 2, times the
    // time step and the 1/n_det of the detector DFT (Eq. FourSerForg).
    std::vector<float> Bi((size_t)(d.K + 1) * (d.J + 1));
    for (int k = 0; k <= d.K; ++k)
      for (int j = 0; j <= d.J; ++j) {
        const double* Jr = &Jt[(size_t)j * KS];
        const double dJ = k == 0 ? -Jr[1] : 0.5 * (Jr[k - 1] - Jr[k + 1]);
        Bi[(size_t)k * (d.J + 1) + j] = (float)(dJ * dt / n_det);
      }
    TAT_TRY(upload(P, Bi, &d.Binv));
    // The same multipliers by ring tile, so that each CTA of the angular stage copies its
    // block with 16-byte asynchronous copies: [tile][k][g], ring 1 + tile*rpc + g.
    {
      const int rpc = rings_per_cta_for(n_phi);
      const int ntiles = (d.J + rpc - 1) / rpc;
      d.bt_bs = ((d.K + 1) * rpc + 3) / 4 * 4;
      std::vector<float> tt((size_t)std::max(ntiles, 1) * d.bt_bs, 0.0f), ti(tt.size(), 0.0f);
      for (int t = 0; t < ntiles; ++t)
        for (int k = 0; k <= d.K; ++k)
          for (int g = 0; g < rpc; ++g) {
            const int rr = 1 + t * rpc + g;
            if (rr > d.J) continue;
            const size_t o = (size_t)t * d.bt_bs + (size_t)k * rpc + g;
            const bool low_zero = low_on && k <= 1 && rr < kLowA;
            tt[o] = low_zero ? 0.0f : Bt[(size_t)k * (d.J + 1) + rr];
            ti[o] = Bi[(size_t)k * (d.J + 1) + rr];
          }
      TAT_TRY(upload(P, tt, &d.Btt));
      TAT_TRY(upload(P, ti, &d.Bit));
    }
    std::vector<float> Bh(2 * std::max(d.n_low, 1), 0.0f), Lc((size_t)std::max(d.n_low, 1) * n_t, 0.0f);
    for (int q = 0; q < d.n_low; ++q) {
      const int r = d.J + 1 + q;
      for (int k = 0; k < 2; ++k)
        Bh[k * d.n_low + q] = (float)(lw[q] * dlam * lam[r] * Jt[(size_t)r * KS + k] / n_phi);
      for (int m = 0; m < n_t; ++m) Lc[(size_t)q * n_t + m] = (float)std::cos(lam[r] * ((double)m * dt));
    }
    TAT_TRY(upload(P, Bh, &d.Bh));
    TAT_TRY(upload(P, Lc, &d.Lcos));
  }
  // Half-circle angles phi_l, l = l' - n_phi/4, l' = 0..nh-1 (phi in [-pi/2, pi/2)).
  std::vector<double> hc(d.nh), hs(d.nh);
  {
    std::vector<float2> cs(d.nh);
    for (int lp = 0; lp < d.nh; ++lp) {
      cos_sin_2pi(lp - n_phi / 4, n_phi, &hc[lp], &hs[lp]);
      cs[lp] = make_float2((float)hc[lp], (float)hs[lp]);
    }
    TAT_TRY(upload(P, cs, &d.cs_half));
  }
  // Inverse (Algorithm 3, step 5): polar position of every node (c, q) of one
  // quadrant of the Cartesian spectrum grid, in FP64 (the other quadrants of
  // the half plane are its mirror q -> -q).  Ring: u = |(c, q)| dxi / dlam,
  // kept up to J + 1e-6 (ties u = J occur exactly when dxi/dlam is rational),
  // j = min(floor(u), J-1), a = u - j; angle: phi = atan2(q, c) in cells of
  // 2pi/n_phi, L = floor, b = the fraction.
  {
    const int h2 = d.N / 2;
    std::vector<unsigned> jl((size_t)h2 * h2);
    std::vector<float2> ab((size_t)h2 * h2);
    std::vector<int> qmax(h2, -1);  // u grows with q along a column: the inside rows are q <= qmax
    const double rho = dxi / dlam, acell = n_phi / (2.0 * kPi);
    parallel_for(h2, [&](int c) {
      for (int q = 0; q < h2; ++q) {
        const size_t e = (size_t)c * h2 + q;
        const double u = std::sqrt((double)c * c + (double)q * q) * rho;
        const double ph = std::atan2((double)q, (double)c) * acell;
        const double Lf = std::floor(ph);
        unsigned j = 0xffffu;
        double a = 0.0;
        if (u <= d.J + 1e-6) {
          const double jf = std::min(std::floor(u), (double)(d.J - 1));
          j = (unsigned)jf;
          a = std::min(u - jf, 1.0);
          qmax[c] = q;
        }
        jl[e] = j | ((unsigned)Lf << 16);
        ab[e] = make_float2((float)a, (float)(ph - Lf));
      }
    });
    TAT_TRY(upload(P, jl, &d.inv_jl));
    TAT_TRY(upload(P, ab, &d.inv_ab));
    TAT_TRY(upload(P, qmax, &d.inv_qmax));
    d.inv_scale = (float)(dxi * dxi / (2.0 * kPi));
    d.inv_ok = n_phi == n_det ? 1 : 0;
  }
  // Bilinear stencils of every half-plane polar sample (rings 1..J and the
  // low-mode rings), bucketed by stencil column i0 and sorted by row k0.
  {
    const int npts = (d.n_rings - 1) * d.nh;
    std::vector<PolarEntry> ent(npts);
    std::vector<int> col(npts);
    int idx = 0;
    for (int r = 1; r < d.n_rings; ++r) {
      for (int lp = 0; lp < d.nh; ++lp) {
        const double u = lam[r] * hc[lp] / dxi;
        const double v = lam[r] * hs[lp] / dxi;
        const double fu = std::floor(u), fv = std::floor(v);
        const long long i0 = (long long)fu, k0 = (long long)fv;
        if (i0 < 0 || i0 > d.ncol - 2 || k0 < -(d.N / 2 - 1) || k0 > d.N / 2 - 2) return TAT_ERR_INTERNAL;
        ent[idx] = PolarEntry{r * d.nh + lp, (int)k0, (float)(u - fu), (float)(v - fv)};
        col[idx] = (int)i0;
        ++idx;
      }
    }
    std::vector<int> off(d.ncol + 1, 0);
    for (int i = 0; i < npts; ++i) off[col[i] + 1]++;
    for (int c = 0; c < d.ncol; ++c) off[c + 1] += off[c];
    std::vector<PolarEntry> sorted(npts);
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int i = 0; i < npts; ++i) sorted[fill[col[i]]++] = ent[i];
    for (int c = 0; c < d.ncol; ++c)
      std::sort(sorted.begin() + off[c], sorted.begin() + off[c + 1], [](const PolarEntry& x, const PolarEntry& y) {
        return x.k0 != y.k0 ? x.k0 < y.k0 : x.p < y.p;
      });
    // Runs of equal stencil row k0 within a column ({first point, k0}), for the
    // adjoint's deterministic scatter; a sentinel {npts, 0} follows the last run,
    // so run r ends where run r + 1 starts.
    std::vector<int2> runs;
    std::vector<int> runoff(d.ncol + 1, 0);
    runs.reserve(npts + 1);
    for (int c = 0; c < d.ncol; ++c) {
      runoff[c] = (int)runs.size();
      for (int e = off[c]; e < off[c + 1]; ++e)
        if (e == off[c] || sorted[e].k0 != sorted[e - 1].k0) runs.push_back(make_int2(e, sorted[e].k0));
    }
    runoff[d.ncol] = (int)runs.size();
    runs.push_back(make_int2(npts, 0));
    std::vector<int> pinv((size_t)d.n_rings * d.nh, -1);
    for (int e = 0; e < npts; ++e) pinv[sorted[e].p] = e;
    for (size_t p = d.nh; p < pinv.size(); ++p)
      if (pinv[p] < 0) return TAT_ERR_INTERNAL;  // every sample of rings >= 1 has exactly one point
    TAT_TRY(upload(P, pinv, &d.pinv));
    TAT_TRY(upload(P, sorted, &d.pts));
    // the split forward column stage's copy of the table (N = 512 RB, few enough rows)
    const bool split_ok = (d.N == 512 || d.N == 1024 || d.N == 2048 || d.N == 4096 || d.N == 8192) &&
                          n <= (d.N == 8192 ? 1024 : 512);
    if (split_ok) {
      const int RB = d.N / 512;
      auto slot = [&](long long q) { return (unsigned)((q % RB) * kSplitRegionSlots + q / RB); };
      std::vector<PolarEntrySplit> ps(npts);
      for (int e = 0; e < npts; ++e) {
        const PolarEntry& s = sorted[e];
        const long long k0 = s.k0, k1 = s.k0 + 1;  // signed rows; |k| < N/2
        double c0, s0, c1, s1;
        cos_sin_2pi(k0 * (n - 1), 2LL * d.N, &c0, &s0);
        cos_sin_2pi(k1 * (n - 1), 2LL * d.N, &c1, &s1);
        const double b = s.b;
        PolarEntrySplit& t = ps[e];
        t.p = s.p;
        t.slots = slot(k0 < 0 ? k0 + d.N : k0) | (slot(k1 < 0 ? k1 + d.N : k1) << 16);
        t.a = s.a;
        t.pad = 0.f;
        t.alpha = make_float2((float)((1.0 - b) * c0), (float)((1.0 - b) * s0));
        t.beta = make_float2((float)(b * c1), (float)(b * s1));
      }
      TAT_TRY(upload(P, ps, &d.pts_split));
    }
    TAT_TRY(upload(P, off, &d.coloff));
    TAT_TRY(upload(P, runs, &d.runs));
    TAT_TRY(upload(P, runoff, &d.runoff));
    if (npts != P->info.n_points) return TAT_ERR_INTERNAL;
  }
  // Launch shapes.
  LaunchCfg& c = P->cfg;
  // Lengths RA*256 (RA = 2..32) use the in-place four-step transform, 256 threads
  // per row pair by default (any multiple of 32 works); up to 4 row pairs (1024
  // threads) per CTA.
  const bool four_step = d.N == 512 || d.N == 1024 || d.N == 2048 || d.N == 4096 || d.N == 8192;
  c.nt_rows = four_step ? std::max(c.nt_N, 256) : c.nt_N;
  // the four-step transform needs groups of at least 64 threads (step B of RA = 4)
  if (d.n_phi == 1024) c.nt_phi = std::max(c.nt_phi, 64);
  if (n_det == 1024) c.nt_det = std::max(c.nt_det, 64);
  c.rows_pairs = d.N == 8192 ? 1 : std::max(1, std::min(4, 1024 / c.nt_rows));
  c.strip = 8;
  c.cols_threads = std::max(c.nt_N, 256);
  // measured at the benchmark sizes: both stages gain at N = 1024 .. 4096; at N = 512 only the
  // forward, at N = 8192 only the adjoint (the autotuner tries every combination)
  if ((d.N == 512 || d.N == 1024 || d.N == 2048 || d.N == 4096 || d.N == 8192) && n <= (d.N == 8192 ? 1024 : 512))
    c.cols_split = d.N == 512 ? 1 : d.N == 8192 ? 2 : 3;
  else
    c.cols_split = 0;
  c.pdl = d.N <= 2048;  // measured: +13 % pairs/s at N = 1024, B = 8; -2 % at N = 4096, B = 32
  c.rings_per_cta = rings_per_cta_for(n_phi);
  c.t_tile = time_tile_for(n_det);
  // Workspace per image (float2): X holds row spectra (n x N/2) or per-mode
  // coefficients ((K+1) x (J+1) + 2 low-mode rows); Y holds polar samples
  // (n_rings x nh) or time modes ((K+1) x n_t).
  auto al = [](size_t x) { return (x + 63) / 64 * 64; };
  P->ws_x = al(std::max((size_t)n * d.ncol, (size_t)(d.K + 1) * (d.J + 1) + 2 * (size_t)std::max(d.n_low, 1)));
  P->ws_y = al(std::max((size_t)d.n_rings * d.nh, (size_t)(d.K + 1) * n_t));
  return TAT_OK;
}

void free_plan(tat_plan_s* P) {
  for (void* p : P->allocations) cudaFree(p);
  P->allocations.clear();
}

}  // namespace tat
