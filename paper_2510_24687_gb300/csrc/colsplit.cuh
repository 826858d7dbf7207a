// Column stages of A and A* for FFT lengths N = 512 RB (RB = 1, 2, 4, 8, 16) with the
// column transform split over the RB warps of a CTA (Algorithm 1 step 2 and its transpose
// in Algorithm 2).
//
// A column holds at most n <= 512 non-zero rows (at RB = 16, up to 1024), so with
// q = k1 + RB k2 (k1 < RB, k2 < 512)
//   X[k1 + RB k2] = sum_{m < 512} u_k1[m] w_512^{m k2},     w_M = e^{-2 pi i / M},
//   u_k1[m] = w_N^{m k1} (x[m] + w_16^{k1} x[m + 512]),  the second term only at RB = 16:
// RB independent 512-point DFTs of differently twiddled copies of the column, one per
// warp.  Warp k1, lane l = l' + 16 p (l' < 16, p < 2) holds u[32 j + l], j < 16:
//   1. u *= w_N^{(32 j + 16 p) k1}                           (shared table, per warp)
//   2. DFT16 over j in registers                            -> a
//   3. u *= w_512^{l a}                                      (powers of a per-lane root)
//   4. radix-2 across the lane pair l, l ^ 16 (warp shuffles), u *= w_32^{l' p} w_N^{l' k1}
//   5. transpose within each half-warp through a warp-private region of the column
//      buffer (rows of 17 slots: conflict-free both ways, immediate offsets)
//   6. DFT16 over l' in registers: lane L = a + 16 r holds X[k1 + RB (L + 32 b)], b < 16.
// Step 3 and the lane constant of step 4 together are w_N^{l (k1 + RB a)}; the factor
// w_N^{16 p k1} of the lane's second half rides on step 1.  The CTA synchronises only
// between whole columns: the transform itself needs __syncwarp alone.
//
// Column buffer: bin q in slot (q mod RB) * kSplitRegion + q / RB -- warp k1's 512
// outputs contiguous in its own region, which is also its transpose scratch (543 slots).
// The adjoint runs the conjugate transpose of steps 6..1 per warp, writes each warp's
// 512 partial rows s_k1[m] into its region, and sums the RB regions in the order
// k1 = 0, 1, ... (deterministic, no atomics).
#pragma once

#include "kernels.cuh"

namespace tat {
namespace {

constexpr int kSplitRegion = kSplitRegionSlots;  // slots per warp region (32 rows of 17)

__host__ __device__ constexpr bool split_length(int L) {
  return L == 512 || L == 1024 || L == 2048 || L == 4096 || L == 8192;
}
// Rows a split column transform of length L takes: 512, and 1024 at L = 8192.
__host__ __device__ constexpr int split_max_rows(int L) { return L == 8192 ? 1024 : 512; }

// Buffer slot of column bin q (0 <= q < 512 RB).
template <int RB>
struct SplitSlot {
  __device__ __forceinline__ int operator()(int q) const { return (q & (RB - 1)) * kSplitRegion + q / RB; }
};

// Per-thread constants of steps 3 and 4 (fixed for the whole kernel: they depend on the
// warp and lane only), from the plan's FP64-built length-N twiddle table.
struct SplitTw {
  float2 v1, v2, v4, v8;  // w_512^{l e}, e = 1, 2, 4, 8
  float2 tb;              // w_32^{l' p} w_N^{l' k1}
};

template <int RB>
__device__ __forceinline__ SplitTw split_twiddles(const float2* __restrict__ tw, int k1, int lane) {
  const int lp = lane & 15, p = lane >> 4;
  SplitTw t;
  t.v1 = __ldg(&tw[RB * lane]);
  t.v2 = __ldg(&tw[2 * RB * lane]);
  t.v4 = __ldg(&tw[4 * RB * lane]);
  t.v8 = __ldg(&tw[8 * RB * lane]);
  t.tb = __ldg(&tw[lp * (k1 + 16 * RB * p)]);
  return t;
}

// Step-1 table TG[k1][p][j] = w_N^{(32 j + 16 p) k1}, k1 < RB, in shared memory.
template <int RB>
__device__ __forceinline__ void load_split_tg(float2* tg, const float2* __restrict__ tw, int tid, int nthr) {
  for (int i = tid; i < 32 * RB; i += nthr) {
    const int k1 = i >> 5, p = (i >> 4) & 1, j = i & 15;
    tg[i] = __ldg(&tw[(32 * j + 16 * p) * k1]);
  }
}

// Step 4's radix-2 butterfly across lanes l and l ^ 16: lane p = 0 keeps the sum, p = 1
// the difference (own value of p = 1 is the second operand).  The 2 x 2 matrix is real
// and symmetric, so the adjoint uses the same butterfly.
__device__ __forceinline__ void split_pair_butterfly(float2* v, int lane) {
  const float s = (lane & 16) ? -1.f : 1.f;
#pragma unroll
  for (int a = 0; a < 16; ++a) {
    const float px = __shfl_xor_sync(0xffffffffu, v[a].x, 16);
    const float py = __shfl_xor_sync(0xffffffffu, v[a].y, 16);
    v[a] = make_float2(fmaf(s, v[a].x, px), fmaf(s, v[a].y, py));
  }
}

// Forward, warp k1: v[j] = u_k1[32 j + lane] on entry without the factor w_N^{m k1} (step 1
// applies it); on exit v[b] = X[k1 + RB (lane + 32 b)].
// `reg` is the warp's region of the column buffer (used as transpose scratch) and `tg`
// its row TG[k1][p] of the step-1 table.
__device__ __forceinline__ void split_dft_fwd(float2* v, float2* reg, const float2* tg, const SplitTw& t,
                                              int lane) {
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = cmul(v[j], tg[j]);
  dft16<false>(v);
  apply_twiddles_given<16, false>(v, t.v1, t.v2, t.v4, t.v8);
  split_pair_butterfly(v, lane);
#pragma unroll
  for (int a = 0; a < 16; ++a) v[a] = cmul(v[a], t.tb);
  // lane (l', p) writes row a + 16 p, column l'; lane L reads row L
  float2* w = reg + 272 * (lane >> 4) + (lane & 15);
#pragma unroll
  for (int a = 0; a < 16; ++a) w[17 * a] = v[a];
  __syncwarp();
  const float2* r = reg + 17 * lane;
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = r[i];
  __syncwarp();
  dft16<false>(v);
}

// Adjoint (conjugate transpose of split_dft_fwd), warp k1: v[b] = Z[k1 + RB (lane + 32 b)]
// on entry; on exit v[j] = s_k1[32 j + lane] = w_N^{-m k1} sum_k2 Z[k1 + RB k2] w_512^{-m k2}
// at m = 32 j + lane.  The caller has read the region into v and not yet written it.
__device__ __forceinline__ void split_dft_adj(float2* v, float2* reg, const float2* tg, const SplitTw& t,
                                              int lane) {
  dft16<true>(v);
  __syncwarp();  // every lane has read its inputs from the region
  float2* w = reg + 17 * lane;
#pragma unroll
  for (int i = 0; i < 16; ++i) w[i] = v[i];
  __syncwarp();
  const float2* r = reg + 272 * (lane >> 4) + (lane & 15);
#pragma unroll
  for (int a = 0; a < 16; ++a) v[a] = r[17 * a];
  __syncwarp();
#pragma unroll
  for (int a = 0; a < 16; ++a) v[a] = cmulc(v[a], t.tb);
  split_pair_butterfly(v, lane);
  apply_twiddles_given<16, true>(v, t.v1, t.v2, t.v4, t.v8);
  dft16<true>(v);
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = cmulc(v[j], tg[j]);
}

// Column CTAs of the split transform: RB warps, compiled for 24 / RB CTAs per SM (24 warps;
// at RB = 16 one CTA of 16 warps).
#define TAT_SPLIT_BOUNDS __launch_bounds__(32 * (L / 512), (L / 512) >= 16 ? 1 : 24 / (L / 512))

// Shared memory of the split column kernels of length N: two column buffers, the step-1
// table and the two-level phase table.
__host__ __device__ inline size_t split_cols_smem(int N, int ph_entries) {
  const size_t rb = (size_t)N / 512;
  return (2 * rb * kSplitRegion + 32 * rb + ph_entries) * sizeof(float2);
}

// Warp k1's inputs for column `col` (rows R[c][0..n)): v[j] = x[m] (+ w_16^{k1} x[m + 512]
// at RB = 16), m = 32 j + lane.
template <int RB>
__device__ __forceinline__ void split_load_column(float2* v, const float2* __restrict__ col, int n, int lane,
                                                  float2 w16) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int m = 32 * j + lane;
    float2 x = m < n ? col[m] : make_float2(0.f, 0.f);
    if constexpr (RB == 16) {
      if (m + 512 < n) {
        const float2 y = col[m + 512];
        x = make_float2(fmaf(w16.x, y.x, fmaf(-w16.y, y.y, x.x)), fmaf(w16.x, y.y, fmaf(w16.y, y.x, x.y)));
      }
    }
    v[j] = x;
  }
}

// Forward column stage (same work and outputs as k_cols_fwd): per strip, the column
// transforms of columns c0..c1 and the bilinear gather of the polar samples whose
// stencil column lies in [c0, c1).  Each warp loads all n rows of the next column into
// its registers (the RB warps read the same rows; L1 serves the repeats) while the CTA
// waits at the barrier and gathers, so the transform starts from registers.
template <int L>
__global__ void TAT_SPLIT_BOUNDS k_cols_fwd_split(DevPlan P, const float2* __restrict__ X, long long xs,
                                                  float2* __restrict__ Y, long long ys, int S, int batch) {
  static_assert(split_length(L), "split column transform: N = 512 RB");
  constexpr int RB = L / 512, CS = RB * kSplitRegion;
  TAT_GRID_DEPENDENCY();
  extern __shared__ float2 sm[];
  int strip, b;
  strip_and_image(batch, &strip, &b);
  float2* slot0 = sm;
  float2* slot1 = sm + CS;
  float2* tg = sm + 2 * CS;
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, k1 = tid >> 5;
  const int c0 = strip * S;
  const int c1 = min(c0 + S, P.ncol - 1);  // owned stencil columns i0 in [c0, c1)
  const int ncols = c1 - c0 + 1;           // spectrum columns c0..c1
  const float2* Xb = X + (size_t)b * xs;
  float2* Yb = Y + (size_t)b * ys;
  const int n = P.n;
  const float2 w16 = RB == 16 ? unit_root<16, false>(k1) : make_float2(1.f, 0.f);
  float2 v[16];
  split_load_column<RB>(v, Xb + (size_t)c0 * n, n, lane, w16);
  load_split_tg<RB>(tg, P.fN.tw, tid, NT);
  const SplitTw t = split_twiddles<RB>(P.fN.tw, k1, lane);
  const float2* tgw = tg + 32 * k1 + 16 * (lane >> 4);
  __syncthreads();
#pragma unroll 1
  for (int cc = 0; cc < ncols; ++cc) {
    float2* buf = (cc & 1) ? slot1 : slot0;
    const int c = c0 + cc;
    // the first polar entry of this thread's gather, loaded before the transform
    const int e0 = cc > 0 ? P.coloff[c - 1] + tid : 0, e1 = cc > 0 ? P.coloff[c] : 0;
    PolarEntrySplit pe0{};
    if (e0 < e1) pe0 = P.pts_split[e0];
    float2* reg = buf + k1 * kSplitRegion;
    split_dft_fwd(v, reg, tgw, t, lane);
#pragma unroll
    for (int i = 0; i < 16; ++i) reg[lane + 32 * i] = v[i];
    // the next column's rows (global memory only) are requested before the barrier, so that
    // their latency overlaps the wait for the other warps' transforms
    if (cc + 1 < ncols) split_load_column<RB>(v, Xb + (size_t)(c + 1) * n, n, lane, w16);
    __syncthreads();
    if (cc > 0) {
      const float2* A = (cc & 1) ? slot0 : slot1;  // column c-1
      const float2* B = buf;                       // column c
      // the stencil rows' slots and phase-weighted row weights come precomputed with the point
      for (int e = e0; e < e1; e += NT) {
        const PolarEntrySplit pe = e == e0 ? pe0 : P.pts_split[e];
        const int qa = (int)(pe.slots & 0xffffu), qb = (int)(pe.slots >> 16);
        const float a = pe.a;
        const float2 va = cadd(cscale(A[qa], 1.f - a), cscale(B[qa], a));
        const float2 vb = cadd(cscale(A[qb], 1.f - a), cscale(B[qb], a));
        Yb[pe.p] = cadd(cmul(va, pe.alpha), cmul(vb, pe.beta));
      }
    }
    __syncthreads();
  }
}

// Adjoint column stage (same work and outputs as k_cols_adj): per owned column, the
// deterministic transposed-bilinear scatter (scatter_column), the split inverse
// transform per warp, and the sum of the RB warps' partial rows, stored as R'[c][0..n)
// (at RB = 16 also rows 512..n-1, the sum weighted by w_16^{-k1}); the sum also clears
// the buffer for the column two ahead.  Three CTA barriers per column: after the
// scatter, after the transforms and after the sum.
template <int L>
__global__ void TAT_SPLIT_BOUNDS k_cols_adj_split(DevPlan P, const float2* __restrict__ Y, long long ys,
                                                  float2* __restrict__ X, long long xs, int S, int batch) {
  static_assert(split_length(L), "split column transform: N = 512 RB");
  constexpr int RB = L / 512, CS = RB * kSplitRegion;
  TAT_GRID_DEPENDENCY();
  extern __shared__ float2 sm[];
  int strip, b;
  strip_and_image(batch, &strip, &b);
  const int N = P.N, n = P.n;
  const int tid = threadIdx.x, NT = blockDim.x, lane = tid & 31, k1 = tid >> 5;
  float2* tg = sm + 2 * CS;
  float2* smph = tg + 32 * RB;
  const int c0 = strip * S;
  const int c1 = min(c0 + S, P.ncol);  // owned columns [c0, c1)
  const float2* Yb = Y + (size_t)b * ys;
  float2* Xb = X + (size_t)b * xs;
  auto slot = [&](int c) { return sm + ((c - c0) & 1) * CS; };
  const SplitSlot<RB> pos;
  load_split_tg<RB>(tg, P.fN.tw, tid, NT);
  load_phase2(smph, P, tid, NT);
  const SplitTw t = split_twiddles<RB>(P.fN.tw, k1, lane);
  const float2* tgw = tg + 32 * k1 + 16 * (lane >> 4);
  RunAhead ahead;  // this thread's first run of the next column to scatter
  run_ahead_record(P, c0 - 1, tid, ahead);
  for (int q = tid; q < 2 * CS; q += NT) sm[q] = make_float2(0.f, 0.f);
  run_ahead_point(P, Yb, ahead);
  __syncthreads();
  // right side of the previous strip's last stencil column
  if (c0 >= 1) scatter_column<L, 1, SplitSlot<RB>>(P, Yb, c0 - 1, nullptr, slot(c0), tid, NT, &ahead, smph, pos);
  run_ahead_record(P, c0, tid, ahead);
  run_ahead_point(P, Yb, ahead);
  __syncthreads();
#pragma unroll 1
  for (int c = c0; c < c1; ++c) {
    float2* cur = slot(c);
    float2* nxt = c + 1 < c1 ? slot(c + 1) : nullptr;
    if (c <= P.ncol - 2) scatter_column<L, 1, SplitSlot<RB>>(P, Yb, c, cur, nxt, tid, NT, &ahead, smph, pos);
    run_ahead_record(P, c + 1 < c1 ? c + 1 : -1, tid, ahead);
    __syncthreads();
    if (c == 0) {
      // Column 0 also receives the mirrored samples of the other half circle:
      // F'(0, q) += conj(F'(0, -q)).
      for (int q = tid; q < N / 2; q += NT) {
        if (q == 0) {
          const float2 s = cur[pos(0)];
          cur[pos(0)] = make_float2(2.f * s.x, 0.f);
        } else {
          const int pa = pos(q), pb = pos(N - q);
          const float2 A = cur[pa], B = cur[pb];
          cur[pa] = cadd_rn(A, cconj(B));
          cur[pb] = cadd_rn(B, cconj(A));
        }
      }
      __syncthreads();
    }
    run_ahead_point(P, Yb, ahead);
    // inverse column transform (conj(phase) already applied by the scatter), per warp
    float2* reg = cur + k1 * kSplitRegion;
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = reg[lane + 32 * i];
    split_dft_adj(v, reg, tgw, t, lane);
#pragma unroll
    for (int j = 0; j < 16; ++j) reg[32 * j + lane] = v[j];
    __syncthreads();
    // R'[c][m] = sum_k1 s_k1[m] for m < n (and R'[c][m + 512] = sum_k1 w_16^{-k1} s_k1[m] at
    // RB = 16); each thread then clears the slots it read, and each warp the 32 slots of its
    // region no one reads, ready for the column two ahead
    float2* col = Xb + (size_t)c * n;  // R'[c][0..n): contiguous
    for (int m = tid; m < 512; m += NT) {
      if (m < n) {
        float2 s = cur[m];
#pragma unroll
        for (int w = 1; w < RB; ++w) s = cadd(s, cur[w * kSplitRegion + m]);
        col[m] = s;
      }
      if constexpr (RB == 16) {
        if (m + 512 < n) {
          float2 s = cur[m];
#pragma unroll
          for (int w = 1; w < 16; ++w) s = cadd(s, cmul(cur[w * kSplitRegion + m], unit_root<16, true>(w)));
          col[m + 512] = s;
        }
      }
#pragma unroll
      for (int w = 0; w < RB; ++w) cur[w * kSplitRegion + m] = make_float2(0.f, 0.f);
    }
    cur[k1 * kSplitRegion + 512 + lane] = make_float2(0.f, 0.f);  // the warp's own 32 pad slots
    __syncthreads();
  }
}

}  // namespace
}  // namespace tat
