// CUDA kernels of the fast forward operator A (Algorithm 1) and its exact
// transpose A* (the stages of Algorithm 2), FP32 on the device.
//
// Forward, per image (workspace X, Y are per-image scratch regions):
//   k_rows_fwd   steps 1-2: zero-extend, row DFT of length N (two real rows
//                per complex FFT), x (h^2/2pi) e^{i q dxi}  -> X = R[iy][q], q < N/2
//   k_cols_fwd   steps 2-3: column DFT of length N per half-plane column, kept
//                in shared memory two columns at a time, x e^{i q dxi}, and the
//                bilinear gather of every polar sample whose stencil lies in
//                that column pair  -> Y = F[ring][l']  (the N x N/2 spectrum
//                never reaches global memory)
//   k_rings_fwd  steps 4-5a: per ring, length-n_phi DFT (Eq. eq3) and the
//                per-mode multiplier i^k dlam lam_j J_k(lam_j)/n_phi
//                -> X = C[k][j]; low-mode rings -> two coefficients per ring
//   k_modes_fwd  step 5b: per mode, cosine sum over j (DCT-I through a
//                length-2M FFT of the even extension, Eq. inverse_cos_tr) plus
//                the clustered low-mode quadrature for k = 0, 1  -> Y = G[k][m]
//   k_theta_fwd  steps 6-7: per time sample, inverse DFT over the modes
//                (Eq. FourSerForg; two time samples per complex FFT), arc mask
//                -> g[d][m]
// Adjoint: the same five kernels transposed, in reverse order; between its angular
// and column stages the polar samples lie in the order of the plan's point table
// (column, then row of the bilinear stencil), which the scatter walks.  Only the
// half plane q_x >= 0 of the spectrum and the half circle phi in [-pi/2, pi/2)
// are processed; the other halves follow from Hermitian symmetry (f real).
#pragma once

#include "pdl.cuh"
#include "fft.cuh"
#include "plan.hpp"

namespace tat {
namespace {

// v * i^k and v * (-i)^k without branches (lanes of a warp hold different k).
__device__ __forceinline__ float2 mul_ipow(float2 v, int k) {
  float2 w = (k & 1) ? make_float2(-v.y, v.x) : v;
  const float s = (k & 2) ? -1.f : 1.f;
  return make_float2(s * w.x, s * w.y);
}
__device__ __forceinline__ float2 mul_mipow(float2 v, int k) {
  float2 w = (k & 1) ? make_float2(v.y, -v.x) : v;
  const float s = (k & 2) ? -1.f : 1.f;
  return make_float2(s * w.x, s * w.y);
}
__device__ __forceinline__ int wrapN(int q, int N) { return q < 0 ? q + N : q; }

// The column phase e^{i q dxi} of FFT bin q from the two-level table staged in shared
// memory (load_phase2): one complex product instead of a global load.
__device__ __forceinline__ void load_phase2(float2* dst, const DevPlan& P, int tid, int nthr) {
  for (int i = tid; i < P.ph_lo + 64; i += nthr) dst[i] = P.phase2[i];
}
__device__ __forceinline__ float2 phase_at(const float2* t, const DevPlan& P, int q) {
  const float2 a = t[q >> 6], b = t[P.ph_lo + (q & 63)];
  float2 v = make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
  if (P.ph_flip && q >= (P.N >> 1)) v = make_float2(-v.x, -v.y);
  return v;
}

// 16-byte asynchronous copy global -> shared (cp.async, completion by wait_group: a
// hardware wait, no spinning).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The angular stage's per-tile multiplier block (bt_bs floats of a tiled table) copied to
// shared memory at `dst` (16-byte aligned) with asynchronous copies; the caller waits
// (cp_async_wait_all + barrier) before reading it.
__device__ __forceinline__ void stage_multipliers(float* dst, const float* tiled, int tile, int bs) {
  const float4* src = reinterpret_cast<const float4*>(tiled + (size_t)tile * bs);
  for (int i = threadIdx.x; i < bs / 4; i += blockDim.x) cp_async16(dst + 4 * i, src + i);
  cp_async_commit();
}
__device__ __forceinline__ float* align16(void* p) {
  return reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
}

// ------------------------------------------------------------------ forward

// Row kernels: up to 1024 threads (4 row pairs); at L = 8192 one row pair of 512
// threads, whose 32-point step A needs the registers of a 512-thread bound.
#define TAT_ROWS_BOUNDS __launch_bounds__(L == 8192 ? 512 : 1024)

template <int L>
__global__ void TAT_ROWS_BOUNDS k_rows_fwd(DevPlan P, const float* __restrict__ f, long long fs,
                                                   float2* __restrict__ X, long long xs, int RP, int nt) {
  TAT_GRID_DEPENDENCY();
  extern __shared__ float2 sm[];
  const int b = blockIdx.y;
  const int g = threadIdx.x / nt, gt = threadIdx.x % nt;
  const int SL = xpad_len(P.N);
  float2* buf = sm + g * SL;
  float2* smtw = sm + RP * SL;  // four-step twiddles
  load_fourstep_tw(smtw, P.fN.fstw, threadIdx.x, blockDim.x);
  const int pair = blockIdx.x * RP + g;
  const int iy1 = 2 * pair, iy2 = 2 * pair + 1;
  const bool v1 = iy1 < P.n, v2 = iy2 < P.n;
  const float* fb = f + (size_t)b * fs;
  const int2 r1 = v1 ? P.rowrange[iy1] : make_int2(0, 0);
  const int2 r2 = v2 ? P.rowrange[iy2] : make_int2(0, 0);
  // only the n leading entries are written: the FFT's first pass reads [0, n)
  for (int ix = gt; ix < P.n; ix += nt) {
    float a = 0.f, c = 0.f;
    if (ix >= r1.x && ix < r1.y) a = fb[(size_t)iy1 * P.n + ix];
    if (ix >= r2.x && ix < r2.y) c = fb[(size_t)iy2 * P.n + ix];
    buf[xpad<L>(ix)] = make_float2(a, c);
  }
  __syncthreads();
  col_fft_fwd<L>(buf, P.fN, smtw, gt, nt, nt, P.n, nullptr);
  // Split the two real rows and store R[q][iy] (column-major); the RP pairs of
  // this CTA are adjacent rows, so consecutive threads write consecutive rows.
  float2* Xb = X + (size_t)b * xs;
  const int pair0 = blockIdx.x * RP;
  // the two rows of a pair are adjacent in R[q][.]: one 16-byte store when aligned
  const bool vec = (P.n & 1) == 0 && (xs & 1) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  for (int e = threadIdx.x; e < P.ncol * RP; e += blockDim.x) {
    const int q = e / RP, gg = e - q * RP;
    const int py1 = 2 * (pair0 + gg);
    if (py1 >= P.n) continue;
    const float2* bg = sm + gg * SL;
    const float2 Z = bg[xpad<L>(colpos<L>(q))];
    const float2 Zc = cconj(bg[xpad<L>(colpos<L>(q == 0 ? 0 : P.N - q))]);
    const float2 x1 = cscale(cadd(Z, Zc), 0.5f);
    const float2 dd = csub(Z, Zc);
    const float2 x2 = make_float2(0.5f * dd.y, -0.5f * dd.x);
    const float2 ph = cscale(P.phase[q], P.h2_2pi);
    float2* col = Xb + (size_t)q * P.n;
    const float2 y1 = cmul(ph, x1), y2 = cmul(ph, x2);
    if (py1 + 1 < P.n && vec) {
      *reinterpret_cast<float4*>(col + py1) = make_float4(y1.x, y1.y, y2.x, y2.y);  // rows py1, py1 + 1
    } else {
      col[py1] = y1;
      if (py1 + 1 < P.n) col[py1 + 1] = y2;
    }
  }
}

// Column kernels: up to 384 threads for the compile-time lengths up to 4096 (512
// otherwise), compiled for two 384-thread CTAs per SM -- the same 80-register budget as
// three CTAs of 256 threads, which is the default shape; 384 lets one pass of the
// adjoint's scatter cover a column's runs (about 370 on average at n = 512).
#define TAT_COLS_BOUNDS_F __launch_bounds__((L > 0 && L <= 4096) ? 384 : 512, (L > 0 && L <= 4096) ? 2 : 1)
#define TAT_COLS_BOUNDS_A __launch_bounds__((L > 0 && L <= 4096) ? 384 : 512, (L > 0 && L <= 4096) ? 2 : 1)

// Column strips are launched strip-major (all images' strip 0 first): the
// strips near q_x = 0 hold up to 7x the average number of polar samples, so
// starting them first keeps them off the kernel's tail.
__device__ __forceinline__ void strip_and_image(int batch, int* strip, int* b) {
  *strip = blockIdx.x / batch;
  *b = blockIdx.x % batch;
}

template <int L>
__global__ void TAT_COLS_BOUNDS_F k_cols_fwd(DevPlan P, const float2* __restrict__ X, long long xs,
                                           float2* __restrict__ Y, long long ys, int S, int nt, int batch) {
  TAT_GRID_DEPENDENCY();
  extern __shared__ float2 sm[];
  int strip, b;
  strip_and_image(batch, &strip, &b);
  const int SL = xpad_len(P.N);
  float2* slot0 = sm;
  float2* slot1 = sm + SL;
  float2* smtw = sm + 2 * SL;  // four-step twiddles
  float2* smph = smtw + kFourStepTw;  // two-level phase table
  const int tid = threadIdx.x, NT = blockDim.x;
  load_fourstep_tw(smtw, P.fN.fstw, tid, NT);
  load_phase2(smph, P, tid, NT);
  const int c0 = strip * S;
  const int c1 = min(c0 + S, P.ncol - 1);  // owned stencil columns i0 in [c0, c1)
  const int ncols = c1 - c0 + 1;           // spectrum columns c0..c1
  const float2* Xb = X + (size_t)b * xs;
  float2* Yb = Y + (size_t)b * ys;
  const int N = P.N;
  // the first PolarEntry of each thread's gather is loaded before the column FFT, so that
  // its latency hides behind the transform; so is the next column's input (up to two rows
  // a thread, else it is read when needed)
  PolarEntry pe0{};
  const bool ahead = P.n <= 2 * NT;
  float2 nx0 = make_float2(0.f, 0.f), nx1 = nx0;
  auto load_ahead = [&](int c) {
    const float2* col = Xb + (size_t)c * P.n;
    if (tid < P.n) nx0 = col[tid];
    if (tid + NT < P.n) nx1 = col[tid + NT];
  };
  if (ahead) load_ahead(c0);
#pragma unroll 1
  for (int cc = 0; cc < ncols; ++cc) {
    float2* buf = (cc & 1) ? slot1 : slot0;
    const int c = c0 + cc;
    if (ahead) {
      if (tid < P.n) buf[xpad<L>(tid)] = nx0;
      if (tid + NT < P.n) buf[xpad<L>(tid + NT)] = nx1;
    } else {
      const float2* col = Xb + (size_t)c * P.n;  // R[c][0..n): contiguous
      for (int iy = tid; iy < P.n; iy += NT) buf[xpad<L>(iy)] = col[iy];
    }
    const int e0 = cc > 0 ? P.coloff[c - 1] + tid : 0, e1 = cc > 0 ? P.coloff[c] : 0;
    if (e0 < e1) pe0 = P.pts[e0];
    __syncthreads();
    if (ahead && cc + 1 < ncols) load_ahead(c + 1);
    // column DFT over the n nonzero rows (the phase e^{i q dxi} of each output
    // row is applied by the gather below)
    col_fft_fwd<L>(buf, P.fN, smtw, tid, NT, nt, P.n, nullptr);
    if (cc > 0) {
      const float2* A = (cc & 1) ? slot0 : slot1;  // column c-1
      const float2* B = buf;                       // column c
      for (int e = e0; e < e1; e += NT) {
        const PolarEntry pe = e == e0 ? pe0 : P.pts[e];
        const int ra = wrapN(pe.k0, N), rb = wrapN(pe.k0 + 1, N);
        const int qa = xpad<L>(colpos<L>(ra)), qb = xpad<L>(colpos<L>(rb));
        const float a = pe.a, bb = pe.b;
        const float2 va = cadd(cscale(A[qa], 1.f - a), cscale(B[qa], a));
        const float2 vb = cadd(cscale(A[qb], 1.f - a), cscale(B[qb], a));
        Yb[pe.p] = cadd(cscale(cmul(va, phase_at(smph, P, ra)), 1.f - bb), cscale(cmul(vb, phase_at(smph, P, rb)), bb));
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) s += red[i];
  return s;  // valid in thread 0
}

template <int L>
__global__ void __launch_bounds__(1024) k_rings_fwd(DevPlan P, const float2* __restrict__ Y, long long ys, float2* __restrict__ X,
                            long long xs, int /*rings per CTA*/, int nt, int ntiles) {
  TAT_GRID_DEPENDENCY();
  constexpr int RPC = rings_per_cta_for(L);
  extern __shared__ float2 sm[];
  const int b = blockIdx.y;
  const float2* Yb = Y + (size_t)b * ys;
  float2* Xb = X + (size_t)b * xs;
  const int J1 = P.J + 1;
  if ((int)blockIdx.x >= ntiles) {
    // Low-mode ring: only k = 0 and k = 1 are needed.  Over the full circle
    // (F(phi + pi) = conj F(phi)):  sum_l F_l = 2 sum_half Re F,
    // sum_l F_l e^{-i phi_l} = 2i sum_half Im F e^{-i phi}.
    float* red = reinterpret_cast<float*>(sm);
    const int q = blockIdx.x - ntiles;
    const int r = P.J + 1 + q;
    float s0 = 0.f, sx = 0.f, sy = 0.f;
    for (int l = threadIdx.x; l < P.nh; l += blockDim.x) {
      const float2 F = Yb[(size_t)r * P.nh + l];
      const float2 cs = P.cs_half[l];
      s0 += F.x;
      sx += F.y * cs.x;
      sy -= F.y * cs.y;
    }
    s0 = block_sum(s0, red);
    sx = block_sum(sx, red + 32);
    sy = block_sum(sy, red + 64);
    if (threadIdx.x == 0) {
      float2* Ch = Xb + (size_t)(P.K + 1) * J1;
      const float2 S0 = make_float2(2.f * s0, 0.f);
      const float2 S1 = make_float2(-2.f * sy, 2.f * sx);  // 2i (sx + i sy)
      Ch[q] = cscale(S0, P.Bh[q]);
      Ch[P.n_low + q] = mul_ipow(cscale(S1, P.Bh[P.n_low + q]), 1);
    }
    return;
  }
  const int g = threadIdx.x / nt, gt = threadIdx.x % nt;
  const int SL = xpad_len(P.n_phi);
  float2* buf = sm + g * SL;
  float2* smptw = sm + RPC * SL;
  float2* smtw = smptw + P.fphi.ptw_len;
  float* smB = align16(smtw + kFourStepTw);  // this tile's multipliers [k][g]
  stage_multipliers(smB, P.Btt, blockIdx.x, P.bt_bs);  // in flight during the loads and the FFTs
  load_pass_tw(smptw, P.fphi, threadIdx.x, blockDim.x);
  load_fourstep_tw(smtw, P.fphi.fstw, threadIdx.x, blockDim.x);
  const int rbase = 1 + blockIdx.x * RPC;
  const int r = rbase + g;
  const bool valid = r <= P.J;
  const int q4 = P.n_phi / 4;
  const float2* Fr = Yb + (size_t)r * P.nh;
  // Each half-circle sample F(l') is read once (16-byte loads, two samples each) and lands
  // at l = l' - n_phi/4 (mod n_phi) and, conjugated, at l' + n_phi/4 (F(phi + pi) = conj F(phi)).
#pragma unroll 4
  for (int i = gt; i < P.nh / 2; i += nt) {
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) w = *reinterpret_cast<const float4*>(Fr + 2 * i);
    const int l0 = 2 * i, l1 = l0 + 1;
    buf[xpad<L>(l0 >= q4 ? l0 - q4 : l0 + 3 * q4)] = make_float2(w.x, w.y);
    buf[xpad<L>(l0 + q4)] = make_float2(w.x, -w.y);
    buf[xpad<L>(l1 >= q4 ? l1 - q4 : l1 + 3 * q4)] = make_float2(w.z, w.w);
    buf[xpad<L>(l1 + q4)] = make_float2(w.z, -w.w);
  }
  __syncthreads();
  if constexpr (FourStep<L>::on) col_fft_fwd<L>(buf, P.fphi, smtw, gt, nt, nt, P.n_phi, nullptr);
  else fft<L, false>(buf, P.fphi, gt, nt, P.n_phi, P.K + 1, nullptr, nullptr, smptw);
  cp_async_wait_all();
  __syncthreads();
  for (int e = threadIdx.x; e < (P.K + 1) * RPC; e += blockDim.x) {
    const int k = e / RPC, gg = e % RPC;
    const int rr = rbase + gg;
    if (rr > P.J) continue;
    Xb[(size_t)k * J1 + rr] = mul_ipow(cscale(sm[gg * SL + xpad<L>(colpos<L>(k))], smB[e]), k);
  }
}

template <int L, int V = 0>
__global__ void __launch_bounds__(1024) k_modes_fwd(DevPlan P, const float2* __restrict__ X, long long xs, float2* __restrict__ Y,
                            long long ys, int nt) {
  TAT_GRID_DEPENDENCY();
  extern __shared__ float2 sm[];
  const int b = blockIdx.y, k = blockIdx.x;
  const int J1 = P.J + 1, L2 = 2 * P.M;
  const float2* Cm = X + (size_t)b * xs + (size_t)k * J1;
  float2* smptw = sm + xpad_len(L2);
  load_pass_tw(smptw, P.f2M, threadIdx.x, blockDim.x);
  float2* G = Y + (size_t)b * ys + (size_t)k * P.n_t;
  const bool low = P.low_on && k <= 1;
  const float2* Ch = X + (size_t)b * xs + (size_t)(P.K + 1) * J1 + (size_t)k * P.n_low;
  if constexpr (L > 0) {
    // the even extension is read straight into the first pass (its zero band is not
    // touched) and each kept output leaves the last pass straight for global memory
    const int J = P.J;
    auto load = [&](int j) -> float2 {
      if (j >= 1 && j <= J) return Cm[j];
      if (j >= L2 - J) return Cm[L2 - j];
      return make_float2(0.f, 0.f);
    };
    auto store = [&](int m, float2 x) {
      float2 v = cscale(x, 0.5f);
      if (low) {
        for (int q = 0; q < P.n_low; ++q) {
          const float c = P.Lcos[(size_t)q * P.n_t + m];
          const float2 ch = Ch[q];
          v.x += c * ch.x;
          v.y += c * ch.y;
        }
      }
      G[m] = v;
    };
    __syncthreads();  // twiddles
    fft_io<L, false, V>(sm, P.f2M, threadIdx.x, nt, P.n_t, load, store, smptw);
  } else {
    for (int j = threadIdx.x; j < L2; j += blockDim.x) {
      float2 v = make_float2(0.f, 0.f);
      if (j >= 1 && j <= P.J) v = Cm[j];
      else if (j >= L2 - P.J) v = Cm[L2 - j];
      sm[xpad<L>(j)] = v;
    }
    __syncthreads();
    fft<L, false, V>(sm, P.f2M, threadIdx.x, nt, L2, P.n_t, nullptr, nullptr, smptw);
    for (int m = threadIdx.x; m < P.n_t; m += blockDim.x) {
      float2 v = cscale(sm[xpad<L>(m)], 0.5f);
      if (low) {
        for (int q = 0; q < P.n_low; ++q) {
          const float c = P.Lcos[(size_t)q * P.n_t + m];
          const float2 ch = Ch[q];
          v.x += c * ch.x;
          v.y += c * ch.y;
        }
      }
      G[m] = v;
    }
  }
}

// Mode sum folded onto detector bin `bin` for time sample m: sum of g_k over
// k in [-K, K) with k = bin (mod n_det); g_{-k} = conj(g_k), g_{-K} = G[K].
__device__ __forceinline__ float2 folded_mode(const DevPlan& P, const float2* G, int bin, int m) {
  if (P.n_phi == P.n_det) return G[(size_t)bin * P.n_t + m];
  float2 acc = make_float2(0.f, 0.f);
  int k = bin;
  while (k - P.n_det >= -P.K) k -= P.n_det;
  for (; k < P.K; k += P.n_det) {
    float2 v;
    if (k >= 0) v = G[(size_t)k * P.n_t + m];
    else if (k == -P.K) v = G[(size_t)P.K * P.n_t + m];
    else v = cconj(G[(size_t)(-k) * P.n_t + m]);
    acc = cadd(acc, v);
  }
  return acc;
}

template <int L>
__global__ void __launch_bounds__(1024) k_theta_fwd(DevPlan P, const float2* __restrict__ Y, long long ys, float* __restrict__ g,
                            long long gs, int /*time tile*/, int nt) {
  TAT_GRID_DEPENDENCY();
  constexpr int TT = time_tile_for(L);
  extern __shared__ float2 sm[];
  const int b = blockIdx.y;
  const int m0 = blockIdx.x * TT;
  const int npair = TT / 2;
  const int SL = xpad_len(P.n_det);
  const int nd = P.n_det;
  const float2* G = Y + (size_t)b * ys;
  float2* smptw = sm + npair * SL;
  float2* smtw = smptw + P.fdet.ptw_len;
  load_pass_tw(smptw, P.fdet, threadIdx.x, blockDim.x);
  load_fourstep_tw(smtw, P.fdet.fstw, threadIdx.x, blockDim.x);
  // 16-byte loads of the time-sample pairs (m1, m2) when the modes are not folded, the tile is
  // whole and every row starts on a 16-byte boundary
  const bool vin = P.n_phi == P.n_det && (P.n_t & 1) == 0 && (ys & 1) == 0 && m0 + TT <= P.n_t &&
                   (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
#pragma unroll 4
  for (int e = threadIdx.x; e < (nd / 2 + 1) * npair; e += blockDim.x) {
    const int bin = e / npair, p = e % npair;
    const int m1 = m0 + 2 * p, m2 = m1 + 1;
    float2 x1, x2;
    if (vin) {
      const float4 v = *reinterpret_cast<const float4*>(G + (size_t)bin * P.n_t + m1);
      x1 = make_float2(v.x, v.y);
      x2 = make_float2(v.z, v.w);
    } else {
      x1 = m1 < P.n_t ? folded_mode(P, G, bin, m1) : make_float2(0.f, 0.f);
      x2 = m2 < P.n_t ? folded_mode(P, G, bin, m2) : make_float2(0.f, 0.f);
    }
    if (bin == 0 || bin == nd / 2) { x1.y = 0.f; x2.y = 0.f; }
    float2* z = sm + p * SL;
    z[xpad<L>(colpos<L>(bin))] = make_float2(x1.x - x2.y, x1.y + x2.x);
    if (bin > 0 && bin < nd / 2) z[xpad<L>(colpos<L>(nd - bin))] = make_float2(x1.x + x2.y, x2.x - x1.y);
  }
  __syncthreads();
  {
    const int gi = threadIdx.x / nt, gt = threadIdx.x % nt;
    if constexpr (FourStep<L>::on) col_fft_inv<L>(sm + gi * SL, P.fdet, smtw, gt, nt, nt, P.n_det, nullptr);
    else fft<L, true>(sm + gi * SL, P.fdet, gt, nt, P.n_det, P.n_det, nullptr, nullptr, smptw);
  }
  float* gb = g + (size_t)b * gs;
  if constexpr (TT % 4 == 0) {
    // 16-byte stores of four time samples (two transforms) per detector when aligned
    if ((P.n_t & 3) == 0 && (gs & 3) == 0 && m0 + TT <= P.n_t && (reinterpret_cast<uintptr_t>(g) & 15) == 0) {
      constexpr int Q = TT / 4;
      for (int e = threadIdx.x; e < nd * Q; e += blockDim.x) {
        const int d = e / Q, q = e - d * Q;
        const float gm = P.gamma[d];
        const float2 z0 = sm[(2 * q) * SL + xpad<L>(d)], z1 = sm[(2 * q + 1) * SL + xpad<L>(d)];
        *reinterpret_cast<float4*>(gb + (size_t)d * P.n_t + m0 + 4 * q) =
            make_float4(gm * z0.x, gm * z0.y, gm * z1.x, gm * z1.y);
      }
      return;
    }
  }
  for (int e = threadIdx.x; e < nd * TT; e += blockDim.x) {
    const int d = e / TT, tt = e % TT;
    const int m = m0 + tt;
    if (m >= P.n_t) continue;
    const float2 z = sm[(tt >> 1) * SL + xpad<L>(d)];
    gb[(size_t)d * P.n_t + m] = P.gamma[d] * ((tt & 1) ? z.y : z.x);
  }
}

// ------------------------------------------------------------------ adjoint

template <int L>
__global__ void __launch_bounds__(1024) k_theta_adj(DevPlan P, const float* __restrict__ g, long long gs, float2* __restrict__ Y,
                            long long ys, int /*time tile*/, int nt) {
  TAT_GRID_DEPENDENCY();
  constexpr int TT = time_tile_for(L);
  extern __shared__ float2 sm[];
  const int b = blockIdx.y;
  const int m0 = blockIdx.x * TT;
  const int SL = xpad_len(P.n_det);
  const int nd = P.n_det;
  const float* gb = g + (size_t)b * gs;
  float2* smptw = sm + (TT / 2) * SL;
  float2* smtw = smptw + P.fdet.ptw_len;
  load_pass_tw(smptw, P.fdet, threadIdx.x, blockDim.x);
  load_fourstep_tw(smtw, P.fdet.fstw, threadIdx.x, blockDim.x);
  bool vec = false;
  if constexpr (TT % 4 == 0)
    vec = (P.n_t & 3) == 0 && (gs & 3) == 0 && m0 + TT <= P.n_t && (reinterpret_cast<uintptr_t>(g) & 15) == 0;
  if (vec) {
    // 16-byte loads: four time samples of one detector, the real and imaginary parts of two
    // transforms
    constexpr int Q = TT >= 4 ? TT / 4 : 1;
#pragma unroll 4
    for (int e = threadIdx.x; e < nd * Q; e += blockDim.x) {
      const int d = e / Q, q = e - d * Q;
      const float4 v = __ldg(reinterpret_cast<const float4*>(gb + (size_t)d * P.n_t + m0) + q);
      const float gm = P.gamma[d];
      sm[(2 * q) * SL + xpad<L>(d)] = make_float2(gm * v.x, gm * v.y);
      sm[(2 * q + 1) * SL + xpad<L>(d)] = make_float2(gm * v.z, gm * v.w);
    }
  } else {
    for (int e = threadIdx.x; e < nd * TT; e += blockDim.x) {
      const int d = e / TT, tt = e % TT;
      const int m = m0 + tt;
      const float v = m < P.n_t ? P.gamma[d] * gb[(size_t)d * P.n_t + m] : 0.f;
      float* z = reinterpret_cast<float*>(sm + (tt >> 1) * SL + xpad<L>(d));
      z[tt & 1] = v;
    }
  }
  __syncthreads();
  {
    const int gi = threadIdx.x / nt, gt = threadIdx.x % nt;
    if constexpr (FourStep<L>::on) col_fft_fwd<L>(sm + gi * SL, P.fdet, smtw, gt, nt, nt, P.n_det, nullptr);
    else fft<L, false>(sm + gi * SL, P.fdet, gt, nt, P.n_det, P.n_det, nullptr, nullptr, smptw);
  }
  float2* Gp = Y + (size_t)b * ys;
  if ((P.n_t & 1) == 0 && (ys & 1) == 0 && m0 + TT <= P.n_t && (reinterpret_cast<uintptr_t>(Y) & 15) == 0) {
    // both time samples of a transform at once: one 16-byte store of two modes' values
    constexpr int NP = TT / 2;
    for (int e = threadIdx.x; e < (P.K + 1) * NP; e += blockDim.x) {
      const int k = e / NP, pp = e - k * NP;
      const int bin = k % nd;
      const float2* z = sm + pp * SL;
      const float2 Z = z[xpad<L>(colpos<L>(bin))];
      const float2 Zc = cconj(z[xpad<L>(colpos<L>(bin == 0 ? 0 : nd - bin))]);
      const float2 s2 = cscale(cadd(Z, Zc), 0.5f);
      const float2 dd = csub(Z, Zc);
      *reinterpret_cast<float4*>(Gp + (size_t)k * P.n_t + m0 + 2 * pp) = make_float4(s2.x, s2.y, 0.5f * dd.y, -0.5f * dd.x);
    }
    return;
  }
  for (int e = threadIdx.x; e < (P.K + 1) * TT; e += blockDim.x) {
    const int k = e / TT, tt = e % TT;
    const int m = m0 + tt;
    if (m >= P.n_t) continue;
    const int bin = k % nd;
    const float2* z = sm + (tt >> 1) * SL;
    const float2 Z = z[xpad<L>(colpos<L>(bin))];
    const float2 Zc = cconj(z[xpad<L>(colpos<L>(bin == 0 ? 0 : nd - bin))]);
    float2 x;
    if (tt & 1) {
      const float2 dd = csub(Z, Zc);
      x = make_float2(0.5f * dd.y, -0.5f * dd.x);
    } else {
      x = cscale(cadd(Z, Zc), 0.5f);
    }
    Gp[(size_t)k * P.n_t + m] = x;
  }
}

template <int L, int V = 0>
__global__ void __launch_bounds__(1024) k_modes_adj(DevPlan P, const float2* __restrict__ Y, long long ys, float2* __restrict__ X,
                            long long xs, int nt) {
  TAT_GRID_DEPENDENCY();
  extern __shared__ float2 sm[];
  const int b = blockIdx.y, k = blockIdx.x;
  const int J1 = P.J + 1, L2 = 2 * P.M;
  const float2* Gp = Y + (size_t)b * ys + (size_t)k * P.n_t;
  float2* smptw = sm + xpad_len(L2);
  load_pass_tw(smptw, P.f2M, threadIdx.x, blockDim.x);
  const float2 g0 = Gp[0];
  float2* Dm = X + (size_t)b * xs + (size_t)k * J1;
  const bool low = P.low_on && k <= 1;
  if constexpr (L > 0) {
    // as in k_modes_fwd: the even extension of the time samples straight into the
    // first pass, the kept outputs j < J + 1 straight out of the last one
    const int nt_ = P.n_t;
    auto load = [&](int j) -> float2 {
      if (j < nt_) return Gp[j];
      if (j > L2 - nt_) return Gp[L2 - j];
      return make_float2(0.f, 0.f);
    };
    auto store = [&](int j, float2 x) {
      float2 v = cscale(cadd(x, g0), 0.5f);
      if (low && j < kLowA) v = make_float2(0.f, 0.f);
      Dm[j] = v;
    };
    __syncthreads();  // twiddles
    fft_io<L, false, V>(sm, P.f2M, threadIdx.x, nt, J1, load, store, smptw);
  } else {
    for (int j = threadIdx.x; j < L2; j += blockDim.x) {
      float2 v = make_float2(0.f, 0.f);
      if (j < P.n_t) v = Gp[j];
      else if (j > L2 - P.n_t) v = Gp[L2 - j];
      sm[xpad<L>(j)] = v;
    }
    __syncthreads();
    fft<L, false, V>(sm, P.f2M, threadIdx.x, nt, L2, P.J + 1, nullptr, nullptr, smptw);
    for (int j = threadIdx.x; j < J1; j += blockDim.x) {
      float2 v = cscale(cadd(sm[xpad<L>(j)], g0), 0.5f);
      if (low && j < kLowA) v = make_float2(0.f, 0.f);
      Dm[j] = v;
    }
  }
  if (low) {
    // Dh[k][q] = sum_m cos(lam_q t_m) g'_k(t_m): one warp per low-mode node.
    float2* Dh = X + (size_t)b * xs + (size_t)(P.K + 1) * J1 + (size_t)k * P.n_low;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = w; q < P.n_low; q += nw) {
      float sx = 0.f, sy = 0.f;
      for (int m = l; m < P.n_t; m += 32) {
        const float c = P.Lcos[(size_t)q * P.n_t + m];
        const float2 v = Gp[m];
        sx += c * v.x;
        sy += c * v.y;
      }
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
      }
      if (l == 0) Dh[q] = make_float2(sx, sy);
    }
  }
}

// INV = false: the adjoint's per-mode multiplier (-i)^k dlam lam_j J_k(lam_j)/n_phi and
// the low-mode rings.  INV = true: the inverse's (Eq. Four_coef_v, see k_modes_inv)
// (-i)^(k+1) J'_k(lam_j) dt/n_det and no low-mode rings.  Rings 1..J are written.
template <int L, bool INV = false>
__global__ void __launch_bounds__(1024) k_rings_adj(DevPlan P, const float2* __restrict__ X, long long xs, float2* __restrict__ Y,
                            long long ys, int /*rings per CTA*/, int nt, int ntiles) {
  TAT_GRID_DEPENDENCY();
  constexpr int RPC = rings_per_cta_for(L);
  extern __shared__ float2 sm[];
  const int b = blockIdx.y;
  const float2* Xb = X + (size_t)b * xs;
  float2* Yb = Y + (size_t)b * ys;
  const int J1 = P.J + 1;
  if (!INV && (int)blockIdx.x >= ntiles) {
    // Low-mode ring: F'(phi) = c0 + c1 e^{i phi} + c_{-1} e^{-i phi}, c_{-1} = -conj(c1).
    const int q = blockIdx.x - ntiles;
    const int r = P.J + 1 + q;
    const float2* Dh = Xb + (size_t)(P.K + 1) * J1;
    const float2 c0 = cscale(Dh[q], P.Bh[q]);
    const float2 c1 = mul_mipow(cscale(Dh[P.n_low + q], P.Bh[P.n_low + q]), 1);
    const float2 cm = make_float2(-c1.x, c1.y);
    for (int l = threadIdx.x; l < P.nh; l += blockDim.x) {
      const float2 cs = P.cs_half[l];
      const float2 e = cs, ec = cconj(cs);
      Yb[__ldg(&P.pinv[(size_t)r * P.nh + l])] = cadd(c0, cadd(cmul(c1, e), cmul(cm, ec)));
    }
    return;
  }
  const int SL = xpad_len(P.n_phi);
  float2* smptw = sm + RPC * SL;
  float2* smtw = smptw + P.fphi.ptw_len;
  load_pass_tw(smptw, P.fphi, threadIdx.x, blockDim.x);
  load_fourstep_tw(smtw, P.fphi.fstw, threadIdx.x, blockDim.x);
  const int rbase = 1 + blockIdx.x * RPC;
  // the multipliers come first here, so they are read straight from this tile's contiguous
  // block of the tiled table, together with the coefficients
  const float* Bb = (INV ? P.Bit : P.Btt) + (size_t)blockIdx.x * P.bt_bs;
  for (int e = threadIdx.x; e < (P.K + 1) * RPC; e += blockDim.x) {
    const int k = e / RPC, gg = e % RPC;
    const int rr = rbase + gg;
    float2 w = make_float2(0.f, 0.f);
    if (rr <= P.J) w = mul_mipow(cscale(Xb[(size_t)k * J1 + rr], __ldg(Bb + e)), INV ? k + 1 : k);
    float2* bg = sm + gg * SL;
    bg[xpad<L>(colpos<L>(k))] = w;
    if (k >= 1 && k < P.K) {
      const float2 wc = cconj(w);
      bg[xpad<L>(colpos<L>(P.n_phi - k))] = (k & 1) ? make_float2(-wc.x, -wc.y) : wc;
    }
  }
  __syncthreads();
  const int g = threadIdx.x / nt, gt = threadIdx.x % nt;
  float2* buf = sm + g * SL;
  if constexpr (FourStep<L>::on) col_fft_inv<L>(buf, P.fphi, smtw, gt, nt, nt, P.n_phi, nullptr);
  else fft<L, true>(buf, P.fphi, gt, nt, P.n_phi, P.n_phi, nullptr, nullptr, smptw);
  if constexpr (INV) {
    // Angle-major output Y[l'][ring] (row length J+1, rings 1..J): the inverse's
    // Cartesian nodes along a column read neighbouring rings at nearly one angle,
    // which this layout makes adjacent.  The CTA's rings go out together, so each
    // angle's run of rings is one contiguous write.
    __syncthreads();
    const int q4 = P.n_phi / 4, J1 = P.J + 1, ng = blockDim.x / nt;
    for (int e = threadIdx.x; e < P.nh * ng; e += blockDim.x) {
      const int l = e / ng, gg = e - l * ng, rr = rbase + gg;
      if (rr > P.J) continue;
      int s = l - q4;
      if (s < 0) s += P.n_phi;
      Yb[(size_t)l * J1 + rr] = sm[gg * SL + xpad<L>(s)];
    }
  } else {
    const int r = rbase + g;
    if (r <= P.J) {
      const int q4 = P.n_phi / 4;
      for (int l = gt; l < P.nh; l += nt) {
        int s = l - q4;
        if (s < 0) s += P.n_phi;
        Yb[__ldg(&P.pinv[(size_t)r * P.nh + l])] = buf[xpad<L>(s)];
      }
    }
  }
}

// Explicitly rounded arithmetic for the adjoint's scatter: the compiler may not fuse
// or reorder these, so every inlined copy of the scatter (and the lane-0 recount of
// a neighbour's sum) performs the same operations and gives the same bits.
__device__ __forceinline__ void acc_rn(float2& acc, float w, float2 v) {
  acc.x = __fmaf_rn(w, v.x, acc.x);
  acc.y = __fmaf_rn(w, v.y, acc.y);
}
__device__ __forceinline__ float2 cadd_rn(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 cmulc_rn(float2 a, float2 b) {  // a * conj(b)
  return make_float2(__fmaf_rn(a.x, b.x, __fmul_rn(a.y, b.y)), __fmaf_rn(a.y, b.x, -__fmul_rn(a.x, b.y)));
}
// bilinear weights (1-a)(1-b), (1-a)b, a(1-b), ab
__device__ __forceinline__ float w_l0(const PolarEntry& e) { return __fmul_rn(__fsub_rn(1.f, e.a), __fsub_rn(1.f, e.b)); }
__device__ __forceinline__ float w_l1(const PolarEntry& e) { return __fmul_rn(__fsub_rn(1.f, e.a), e.b); }
__device__ __forceinline__ float w_r0(const PolarEntry& e) { return __fmul_rn(e.a, __fsub_rn(1.f, e.b)); }
__device__ __forceinline__ float w_r1(const PolarEntry& e) { return __fmul_rn(e.a, e.b); }

// A thread's first run of a column (run runoff[c] + tid), loaded ahead of the column's
// scatter in two steps -- run record, then its first point and polar sample (the
// samples lie in the order of the point table, so both come from the run's first
// index) -- each issued a phase before it is needed, so that the column transform in
// between hides the latency of the dependent global loads.
struct RunAhead {
  int s = -1, e = 0, k = 0;  // first point, end, key (s < 0: no run for this thread)
  bool prev = false, next = false;  // runs with keys k-1 / k+1 in the same column
  PolarEntry pe{};
  float2 v = make_float2(0.f, 0.f);
};

// (run runoff[c] + tid + off: off = i * NT for the thread's run of scatter batch i)
__device__ __forceinline__ void run_ahead_record(const DevPlan& P, int c, int tid, RunAhead& q, int off = 0) {
  q.s = -1;
  if (c < 0 || c > P.ncol - 2) return;
  const int r0 = P.runoff[c], r1 = P.runoff[c + 1], r = r0 + tid + off;
  if (r >= r1) return;
  const int2 run = P.runs[r], nx = P.runs[r + 1];
  const int pk = r > r0 ? P.runs[r - 1].y : 0;
  q.s = run.x;
  q.e = nx.x;
  q.k = run.y;
  q.prev = r > r0 && pk == run.y - 1;
  q.next = r + 1 < r1 && nx.y == run.y + 1;
}
__device__ __forceinline__ void run_ahead_point(const DevPlan& P, const float2* __restrict__ Yb, RunAhead& q) {
  if (q.s >= 0) {
    q.pe = P.pts[q.s];
    q.v = Yb[q.s];
  }
}

// Transposed bilinear weights of the points with stencil column i0 = c, added
// into the column buffers of c (weight 1-a) and c+1 (weight a); either may be
// null.  The sum is the same on every call, bit for bit: each run of points
// with one stencil row k0 (the plan's run table) is summed by one lane, in the
// table's order, into its row-k0 part (weight 1-b) and row-k0+1 part (weight b),
// and every buffer cell is written by exactly one lane with a plain add --
// cell k0 by the run with key k0, which first adds the row-k0 part of the run
// with key k0-1 if there is one, and cell k0+1 by the run with key k0 when no
// run has key k0+1.  No atomics: the order of every addition is fixed.
// The conj(phase) of the column transform is applied once per cell.  `qa[i]`,
// i < NA, hold this thread's runs of the column's first NA batches (run
// runoff[c] + tid + i * NT), loaded ahead (RunAhead).
// Buffer slot of column bin q in the four-step column layout (padded, permuted).
template <int L>
struct ColSlot {
  __device__ __forceinline__ int operator()(int q) const { return xpad<L>(colpos<L>(q)); }
};

template <int L, int NA = 1, class Slot = ColSlot<L>>
__device__ __forceinline__ void scatter_column(const DevPlan& P, const float2* __restrict__ Yb, int c, float2* left,
                                               float2* right, int tid, int NT, const RunAhead* qa,
                                               const float2* smph, Slot slot = Slot{}) {
  const unsigned full = 0xffffffffu;
  const int lane = tid & 31;
  const int r0 = P.runoff[c], r1 = P.runoff[c + 1];
  int batch = 0;
  // warp-uniform loop (NT is a multiple of 32): lane l takes run base + l
  for (int base = r0 + (tid - lane); base < r1; base += NT, ++batch) {
    const bool first = batch < NA;
    const RunAhead& q = qa[first ? batch : 0];
    const int r = base + lane;
    const bool valid = r < r1;
    int k = 0, s = 0;
    bool has_prev = false, has_next = false;
    float2 la = make_float2(0.f, 0.f), lb = la, ra = la, rb = la;
    auto add = [&](const PolarEntry& pe, float2 v) {
      acc_rn(la, w_l0(pe), v);
      acc_rn(lb, w_l1(pe), v);
      acc_rn(ra, w_r0(pe), v);
      acc_rn(rb, w_r1(pe), v);
    };
    if (valid) {
      int e;
      if (first) {  // r = r0 + tid + batch * NT: a run loaded ahead
        k = q.k;
        s = q.s;
        e = q.e;
        has_prev = q.prev;
        has_next = q.next;
        add(q.pe, q.v);
        for (int i = s + 1; i < e; ++i) add(P.pts[i], Yb[i]);
      } else {
        const int2 run = P.runs[r], nx = P.runs[r + 1];
        k = run.y;
        s = run.x;
        e = nx.x;
        has_prev = P.runs[r - 1].y == k - 1;  // r > r0 here
        has_next = r + 1 < r1 && nx.y == k + 1;
        for (int i = s; i < e; ++i) add(P.pts[i], Yb[i]);
      }
    }
    // row-k parts of the run with key k-1: from the lane before, or (lane 0) summed again
    float2 plb, prb;
    plb.x = __shfl_up_sync(full, lb.x, 1);
    plb.y = __shfl_up_sync(full, lb.y, 1);
    prb.x = __shfl_up_sync(full, rb.x, 1);
    prb.y = __shfl_up_sync(full, rb.y, 1);
    if (!valid) continue;
    if (has_prev && lane == 0) {
      plb = make_float2(0.f, 0.f);
      prb = plb;
      for (int i = P.runs[r - 1].x; i < s; ++i) {
        const PolarEntry pe = P.pts[i];
        const float2 v = Yb[i];
        acc_rn(plb, w_l1(pe), v);
        acc_rn(prb, w_r1(pe), v);
      }
    }
    const int ra_row = wrapN(k, P.N), rb_row = wrapN(k + 1, P.N);
    const int qa = slot(ra_row), qb = slot(rb_row);
    const float2 pa = phase_at(smph, P, ra_row);
    if (has_prev) {
      la = cadd_rn(la, plb);
      ra = cadd_rn(ra, prb);
    }
    if (left != nullptr) left[qa] = cadd_rn(left[qa], cmulc_rn(la, pa));
    if (right != nullptr) right[qa] = cadd_rn(right[qa], cmulc_rn(ra, pa));
    if (!has_next) {
      const float2 pb = phase_at(smph, P, rb_row);
      if (left != nullptr) left[qb] = cadd_rn(left[qb], cmulc_rn(lb, pb));
      if (right != nullptr) right[qb] = cadd_rn(right[qb], cmulc_rn(rb, pb));
    }
  }
}

template <int L>
__global__ void TAT_COLS_BOUNDS_A k_cols_adj(DevPlan P, const float2* __restrict__ Y, long long ys,
                                           float2* __restrict__ X, long long xs, int S, int nt, int batch) {
  TAT_GRID_DEPENDENCY();
  extern __shared__ float2 sm[];
  int strip, b;
  strip_and_image(batch, &strip, &b);
  const int N = P.N;
  const int SL = xpad_len(N);
  const int tid = threadIdx.x, NT = blockDim.x;
  float2* smtw = sm + 2 * SL;  // four-step twiddles
  float2* smph = smtw + kFourStepTw;  // two-level phase table
  load_fourstep_tw(smtw, P.fN.fstw, tid, NT);
  load_phase2(smph, P, tid, NT);
  const int c0 = strip * S;
  const int c1 = min(c0 + S, P.ncol);  // owned columns [c0, c1)
  const float2* Yb = Y + (size_t)b * ys;
  float2* Xb = X + (size_t)b * xs;
  auto slot = [&](int c) { return sm + ((c - c0) & 1) * SL; };
  RunAhead ahead;  // this thread's first run of the next column to scatter
  {
    float2* first = slot(c0);
    run_ahead_record(P, c0 - 1, tid, ahead);
    for (int q = tid; q < SL; q += NT) first[q] = make_float2(0.f, 0.f);
    run_ahead_point(P, Yb, ahead);
    __syncthreads();
    if (c0 >= 1) scatter_column<L>(P, Yb, c0 - 1, nullptr, first, tid, NT, &ahead, smph);  // right side of the previous column
    run_ahead_record(P, c0, tid, ahead);
    run_ahead_point(P, Yb, ahead);
  }
#pragma unroll 1
  for (int c = c0; c < c1; ++c) {
    float2* cur = slot(c);
    float2* nxt = c + 1 < c1 ? slot(c + 1) : nullptr;
    if (nxt != nullptr)
      for (int q = tid; q < SL; q += NT) nxt[q] = make_float2(0.f, 0.f);
    __syncthreads();
    if (c <= P.ncol - 2) scatter_column<L>(P, Yb, c, cur, nxt, tid, NT, &ahead, smph);
    // the next column's first runs: record now, point and sample before the transform
    run_ahead_record(P, c + 1 < c1 ? c + 1 : -1, tid, ahead);
    __syncthreads();
    if (c == 0) {
      // Column 0 also receives the mirrored samples of the other half circle:
      // F'(0, q) += conj(F'(0, -q)).
      for (int q = tid; q < N / 2; q += NT) {
        if (q == 0) {
          const int p0 = xpad<L>(colpos<L>(0));
          const float2 s = cur[p0];
          cur[p0] = make_float2(2.f * s.x, 0.f);
        } else {
          const int pa = xpad<L>(colpos<L>(q)), pb = xpad<L>(colpos<L>(N - q));
          const float2 A = cur[pa], B = cur[pb];
          cur[pa] = cadd_rn(A, cconj(B));
          cur[pb] = cadd_rn(B, cconj(A));
        }
      }
      __syncthreads();
    }
    // inverse column DFT (conj(phase) already applied by the scatter), first n rows only
    run_ahead_point(P, Yb, ahead);
    col_fft_inv<L>(cur, P.fN, smtw, tid, NT, nt, P.n, nullptr);
    float2* col = Xb + (size_t)c * P.n;  // R'[c][0..n): contiguous
    for (int iy = tid; iy < P.n; iy += NT) col[iy] = cur[xpad<L>(iy)];
    __syncthreads();
  }
}

// Row stage of A* and A^{-1}: rebuilds the Hermitian row spectra of this CTA's
// RP row pairs from the column-major R'[q][iy] and runs the inverse row DFTs;
// row pair g of the CTA ends in sm + g * xpad_len(N), rows 2*pair and 2*pair+1
// in the real and imaginary parts.
template <int L>
__device__ __forceinline__ void rows_inverse_dft(const DevPlan& P, const float2* __restrict__ Xb, float2* sm, int RP,
                                                 int nt) {
  const int g = threadIdx.x / nt, gt = threadIdx.x % nt;
  const int N = P.N;
  const int SL = xpad_len(N);
  float2* buf = sm + g * SL;
  float2* smtw = sm + RP * SL;  // four-step twiddles
  load_fourstep_tw(smtw, P.fN.fstw, threadIdx.x, blockDim.x);
  // Rebuild each row's Hermitian spectrum from R'[q][iy] (column-major):
  // H[q] = conj(phase[q]) R'[q] for q < N/2, H[N-q] = conj(H[q]), H[N/2] = 0;
  // consecutive threads read consecutive rows of one column.
  const int pair0 = blockIdx.x * RP;
  // the two rows of a pair are adjacent in R'[q][.]: one 16-byte load when aligned
  const bool vec = (P.n & 1) == 0 && (reinterpret_cast<uintptr_t>(Xb) & 15) == 0;
#pragma unroll 4
  for (int e = threadIdx.x; e < P.ncol * RP; e += blockDim.x) {
    const int q = e / RP, gg = e - q * RP;
    const int py1 = 2 * (pair0 + gg);
    float2* bg = sm + gg * SL;
    const float2* col = Xb + (size_t)q * P.n;
    float2 r1 = make_float2(0.f, 0.f), r2 = r1;
    if (vec && py1 < P.n) {
      const float4 w = *reinterpret_cast<const float4*>(col + py1);
      r1 = make_float2(w.x, w.y);
      r2 = make_float2(w.z, w.w);
    } else {
      if (py1 < P.n) r1 = col[py1];
      if (py1 + 1 < P.n) r2 = col[py1 + 1];
    }
    const float2 phq = __ldg(&P.phase[q]);
    float2 h1 = py1 < P.n ? cmulc(r1, phq) : make_float2(0.f, 0.f);
    float2 h2 = py1 + 1 < P.n ? cmulc(r2, phq) : make_float2(0.f, 0.f);
    if (q == 0) { h1.y = 0.f; h2.y = 0.f; }
    bg[xpad<L>(colpos<L>(q))] = make_float2(h1.x - h2.y, h1.y + h2.x);
    if (q > 0) bg[xpad<L>(colpos<L>(N - q))] = make_float2(h1.x + h2.y, h2.x - h1.y);  // conj(h1) + i conj(h2)
    else bg[xpad<L>(colpos<L>(N / 2))] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  col_fft_inv<L>(buf, P.fN, smtw, gt, nt, nt, P.n, nullptr);
}

template <int L>
__global__ void TAT_ROWS_BOUNDS k_rows_adj(DevPlan P, const float2* __restrict__ X, long long xs, float* __restrict__ f,
                           long long fs, int RP, int nt) {
  TAT_GRID_DEPENDENCY();
  extern __shared__ float2 sm[];
  const int b = blockIdx.y;
  const int g = threadIdx.x / nt, gt = threadIdx.x % nt;
  rows_inverse_dft<L>(P, X + (size_t)b * xs, sm, RP, nt);
  const float2* buf = sm + g * xpad_len(P.N);
  const int pair = blockIdx.x * RP + g;
  const int iy1 = 2 * pair, iy2 = 2 * pair + 1;
  const bool v1 = iy1 < P.n, v2 = iy2 < P.n;
  float* fb = f + (size_t)b * fs;
  const int2 r1 = v1 ? P.rowrange[iy1] : make_int2(0, 0);
  const int2 r2 = v2 ? P.rowrange[iy2] : make_int2(0, 0);
  for (int ix = gt; ix < P.n; ix += nt) {
    const float2 z = buf[xpad<L>(ix)];
    if (v1) fb[(size_t)iy1 * P.n + ix] = (ix >= r1.x && ix < r1.y) ? P.adj_scale * z.x : 0.f;
    if (v2) fb[(size_t)iy2 * P.n + ix] = (ix >= r2.x && ix < r2.y) ? P.adj_scale * z.y : 0.f;
  }
}

// ------------------------------------------------------------------ inverse (Algorithm 3)
//
// v(x) = F^{-1}[ sum_k e^{ik phi} vhat_k(lambda) ](x), with
//   vhat_k(lambda) = -2 (-i)^|k| J'_|k|(lambda) int_0^T g_k(t) sin(lambda t) dt
// (Eq. Four_coef_v; the constant is fixed by the Fourier transform of G that
// Eq. green_conv and Eq. gseries use), then f = Pi_Omega0 (v + C) with C such
// that v + C has zero mean over Omega \ Omega0 (Eq. silly_integral).  Stages:
// k_theta_adj (g'_k(t_m) = sum_d g e^{-ik theta_d} = n_det g_k), k_modes_inv,
// k_rings_adj<L, true>, k_cols_inv, k_rows_inv, k_inv_finish.

// Sine transform per mode (Algorithm 3, step 3): the length-2M FFT of the odd
// extension of the trapezoid-weighted samples (weight 1/2 at t = T; t = 0 drops
// out) gives FFT_j = -2i sum_m w_m sin(lam_j t_m) g'_k(t_m).  The factor i/2 and
// the -2 of Eq. Four_coef_v make the ring multiplier (-i)^(k+1) J'_k dt/n_det.
template <int L, int V = 0>
__global__ void __launch_bounds__(1024) k_modes_inv(DevPlan P, const float2* __restrict__ Y, long long ys,
                                                    float2* __restrict__ X, long long xs, int nt) {
  TAT_GRID_DEPENDENCY();
  extern __shared__ float2 sm[];
  const int b = blockIdx.y, k = blockIdx.x;
  const int J1 = P.J + 1, L2 = 2 * P.M;
  const float2* Gp = Y + (size_t)b * ys + (size_t)k * P.n_t;
  float2* smptw = sm + xpad_len(L2);
  load_pass_tw(smptw, P.f2M, threadIdx.x, blockDim.x);
  float2* Dm = X + (size_t)b * xs + (size_t)k * J1;
  auto load = [&](int j) -> float2 {
    float2 v = make_float2(0.f, 0.f);
    const int m = j <= P.M ? j : L2 - j;
    if (m > 0 && m < P.n_t) {
      v = Gp[m];
      if (m == P.n_t - 1) v = cscale(v, 0.5f);
      if (j > P.M) v = make_float2(-v.x, -v.y);
    }
    return v;
  };
  if constexpr (L > 0) {
    // the odd extension straight into the first pass, the kept outputs straight out
    auto store = [&](int j, float2 x) { Dm[j] = x; };
    __syncthreads();  // twiddles
    fft_io<L, false, V>(sm, P.f2M, threadIdx.x, nt, J1, load, store, smptw);
  } else {
    for (int j = threadIdx.x; j < L2; j += blockDim.x) sm[xpad<L>(j)] = load(j);
    __syncthreads();
    fft<L, false, V>(sm, P.f2M, threadIdx.x, nt, L2, J1, nullptr, nullptr, smptw);
    for (int j = threadIdx.x; j < J1; j += blockDim.x) Dm[j] = sm[xpad<L>(j)];
  }
}

// Polar sample (ring j, angle l') of the half circle from the angle-major
// Y[l'][j] that k_rings_adj<L, true> writes; ring 0 (lambda = 0) is zero for the
// inverse, and l' = nh (phi = pi/2) is the conjugate of l' = 0 (phi = -pi/2).
__device__ __forceinline__ float2 inv_polar(const DevPlan& P, const float2* __restrict__ Yb, int j, int l) {
  if (j == 0) return make_float2(0.f, 0.f);
  const size_t J1 = (size_t)P.J + 1;
  if (l >= P.nh) return cconj(Yb[(size_t)(l - P.nh) * J1 + j]);
  return Yb[(size_t)l * J1 + j];
}

// vhat at the Cartesian node (c, qs) of the half plane (Algorithm 3, step 5):
// bilinear interpolation in (lambda, phi) of the polar samples, zero beyond
// the cut-off.  The node's ring and angle positions come from the plan's FP64
// quadrant table (an FP32 position would be off by ~1e-4 of a cell at the
// outer rings, which the interpolation weights would carry); qs < 0 is the
// mirror phi -> -phi of |qs|.  Half-circle angle cell: l' = nh/2 + phi cells.
__device__ __forceinline__ float2 inv_node(const DevPlan& P, const float2* __restrict__ Yb, int c, int qs) {
  const int h2 = P.N >> 1;
  const int aq = qs < 0 ? -qs : qs;
  if (aq >= h2) return make_float2(0.f, 0.f);  // the Nyquist row lies beyond the cut-off
  const size_t e = (size_t)c * h2 + aq;
  const unsigned jl = __ldg(&P.inv_jl[e]);
  const int j = (int)(jl & 0xffffu);
  if (j == 0xffff) return make_float2(0.f, 0.f);
  const float2 ab = __ldg(&P.inv_ab[e]);
  const int L = (int)(jl >> 16);
  int l0;
  float bb;
  if (qs >= 0) {
    l0 = (P.nh >> 1) + L;
    bb = ab.y;
  } else if (ab.y > 0.f) {
    l0 = (P.nh >> 1) - L - 1;
    bb = 1.f - ab.y;
  } else {
    l0 = (P.nh >> 1) - L;
    bb = 0.f;
  }
  if (l0 >= P.nh) {  // phi = pi/2 exactly
    l0 = P.nh - 1;
    bb = 1.f;
  }
  const float a = ab.x;
  const float2 v00 = inv_polar(P, Yb, j, l0), v01 = inv_polar(P, Yb, j, l0 + 1);
  const float2 v10 = inv_polar(P, Yb, j + 1, l0), v11 = inv_polar(P, Yb, j + 1, l0 + 1);
  const float2 va = cadd(cscale(v00, 1.f - bb), cscale(v01, bb));
  const float2 vb = cadd(cscale(v10, 1.f - bb), cscale(v11, bb));
  return cadd(cscale(va, 1.f - a), cscale(vb, a));
}

// Steps 5-6 (columns): per strip of half-plane columns, vhat on the whole
// column (times conj(e^{i q dxi}), the x_0 = -1 phase of the inverse DFT), the
// inverse column DFT, first n rows kept -> X = V'[c][iy].
#define TAT_COLS_BOUNDS_I __launch_bounds__((L > 0 && L <= 4096) ? 256 : 512, (L > 0 && L <= 4096) ? 4 : 1)

template <int L>
__global__ void TAT_COLS_BOUNDS_I k_cols_inv(DevPlan P, const float2* __restrict__ Y, long long ys,
                                           float2* __restrict__ X, long long xs, int S, int nt, int batch) {
  TAT_GRID_DEPENDENCY();
  extern __shared__ float2 sm[];
  int strip, b;
  strip_and_image(batch, &strip, &b);
  const int N = P.N;
  const int SL = xpad_len(N);
  const int tid = threadIdx.x, NT = blockDim.x;
  float2* buf = sm;
  float2* smtw = sm + SL;  // four-step twiddles
  load_fourstep_tw(smtw, P.fN.fstw, tid, NT);
  const int c0 = strip * S;
  const int c1 = min(c0 + S, P.ncol);
  const float2* Yb = Y + (size_t)b * ys;
  float2* Xb = X + (size_t)b * xs;
#pragma unroll 1
  for (int c = c0; c < c1; ++c) {
    const int qmax = P.inv_qmax[c];  // rows beyond it lie outside the cut-off: zero, no table read
    for (int q = tid; q < N; q += NT) {
      const int qs = q < N / 2 ? q : q - N;
      const float2 v = (qs <= qmax && -qs <= qmax) ? inv_node(P, Yb, c, qs) : make_float2(0.f, 0.f);
      buf[xpad<L>(colpos<L>(q))] = cmulc(v, __ldg(&P.phase[q]));
    }
    __syncthreads();
    col_fft_inv<L>(buf, P.fN, smtw, tid, NT, nt, P.n, nullptr);
    float2* col = Xb + (size_t)c * P.n;
    for (int iy = tid; iy < P.n; iy += NT) col[iy] = buf[xpad<L>(iy)];
    __syncthreads();
  }
}

// Steps 6 (rows) and 7: the inverse row DFTs give v on the whole n x n grid
// (times dxi^2/2pi); each CTA adds its sum of v over Omega \ Omega0 into the
// image's accumulator.
template <int L>
__global__ void TAT_ROWS_BOUNDS k_rows_inv(DevPlan P, const float2* __restrict__ X, long long xs,
                                                   float* __restrict__ f, long long fs, float* acc, long long accs,
                                                   int RP, int nt) {
  TAT_GRID_DEPENDENCY();
  extern __shared__ float2 sm[];
  const int b = blockIdx.y;
  const int g = threadIdx.x / nt, gt = threadIdx.x % nt;
  rows_inverse_dft<L>(P, X + (size_t)b * xs, sm, RP, nt);
  const float2* buf = sm + g * xpad_len(P.N);
  const int pair = blockIdx.x * RP + g;
  const int iy1 = 2 * pair, iy2 = 2 * pair + 1;
  const bool v1 = iy1 < P.n, v2 = iy2 < P.n;
  float* fb = f + (size_t)b * fs;
  const int2 s1 = v1 ? P.rowrange[iy1] : make_int2(0, 0), o1 = v1 ? P.outrange[iy1] : make_int2(0, 0);
  const int2 s2 = v2 ? P.rowrange[iy2] : make_int2(0, 0), o2 = v2 ? P.outrange[iy2] : make_int2(0, 0);
  float ring = 0.f;
  for (int ix = gt; ix < P.n; ix += nt) {
    const float2 z = buf[xpad<L>(ix)];
    const float a = P.inv_scale * z.x, c = P.inv_scale * z.y;
    if (v1) {
      fb[(size_t)iy1 * P.n + ix] = a;
      if (ix >= o1.x && ix < o1.y && !(ix >= s1.x && ix < s1.y)) ring += a;
    }
    if (v2) {
      fb[(size_t)iy2 * P.n + ix] = c;
      if (ix >= o2.x && ix < o2.y && !(ix >= s2.x && ix < s2.y)) ring += c;
    }
  }
  // block sum in shared memory (the block need not be a multiple of 32 threads)
  __syncthreads();
  float* red = reinterpret_cast<float*>(sm);
  red[threadIdx.x] = ring;
  __syncthreads();
  for (int st = 1; st < (int)blockDim.x; st <<= 1) {
    if ((threadIdx.x & (2 * st - 1)) == 0 && threadIdx.x + st < blockDim.x) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) acc[(size_t)b * accs + 1 + blockIdx.x] = red[0];  // this CTA's partial sum
}

// The sum over Omega \ Omega0 of each image from its row CTAs' `nblk` partial sums (slots
// 1..nblk after the accumulator), in a fixed order -- each thread a fixed set of slots,
// then a fixed tree -- so that A^-1 gives the same bits on every call; one CTA per image.
__global__ void k_inv_sum(int nblk, float* acc, long long accs) {
  TAT_GRID_DEPENDENCY();
  __shared__ float red[256];
  float* a = acc + (size_t)blockIdx.x * accs;
  float s = 0.f;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += a[1 + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) a[0] = red[0];
}

// Step 8: f = Pi_Omega0 (v + C), C = -(sum of v over Omega \ Omega0) / (its node count).
__global__ void k_inv_finish(DevPlan P, int batch, const float* __restrict__ acc, long long accs, float* f,
                             long long fs) {
  TAT_GRID_DEPENDENCY();
  const long long nn = (long long)P.n * P.n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn * batch;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / nn, r = i - b * nn;
    const int iy = (int)(r / P.n), ix = (int)(r - (long long)iy * P.n);
    const float C = P.inv_count > 0.f ? -acc[(size_t)b * accs] / P.inv_count : 0.f;
    const int2 s = P.rowrange[iy];
    float* p = f + (size_t)b * fs + r;
    *p = (ix >= s.x && ix < s.y) ? *p + C : 0.f;
  }
}

}  // namespace
}  // namespace tat
