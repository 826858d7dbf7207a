// Launch shapes and FFT-length dispatch shared by the forward and adjoint
// launchers.  Each kernel is instantiated for the FFT lengths of the common
// problem sizes (compile-time pass schedule) plus a runtime-length fallback.
#pragma once

#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "kernels.cuh"
#include "colsplit.cuh"

namespace tat {
namespace {

struct Shapes {
  dim3 rows_grid, cols_grid_f, cols_grid_a, cols_grid_i, rings_grid, modes_grid, theta_grid;
  int strip_i;  // columns per CTA of A^-1's column stage
  int rows_block, cols_block, cols_block_i, rings_block, modes_block, theta_block;
  size_t rows_smem, cols_smem_f, cols_smem_a, cols_smem_i, rings_smem, modes_smem, theta_smem;
  int ntiles;
  bool cols_split_f, cols_split_a;  // the forward / adjoint column stage on the warp-split transform
  int cols_block_split;              // CTA size of the split column kernels: one warp per 512 points
};

inline Shapes shapes(const tat_plan_s* Pl, int batch) {
  const DevPlan& P = Pl->d;
  const LaunchCfg& c = Pl->cfg;
  Shapes s;
  const int npairs = (P.n + 1) / 2;
  s.rows_grid = dim3((npairs + c.rows_pairs - 1) / c.rows_pairs, batch);
  s.rows_block = c.rows_pairs * c.nt_rows;
  s.rows_smem = ((size_t)c.rows_pairs * xpad_len(P.N) + kFourStepTw) * sizeof(float2);
  // 1-D, strip-major: blockIdx.x = strip * batch + image
  s.cols_grid_f = dim3(((P.ncol - 1 + c.strip - 1) / c.strip) * batch);
  s.cols_grid_a = dim3(((P.ncol + c.strip - 1) / c.strip) * batch);
  // A^-1's gather-bound column stage is fastest with short strips (measured at n = 256, 512:
  // 8 columns ahead of 16 and 32), whatever the pair's tuned strip
  s.strip_i = std::min(c.strip, 8);
  s.cols_grid_i = dim3(((P.ncol + s.strip_i - 1) / s.strip_i) * batch);
  s.cols_block = c.cols_threads;
  // the inverse's column kernel is compiled for at most 256 threads at these lengths
  const bool ct_le4096 = P.N == 256 || P.N == 512 || P.N == 1024 || P.N == 2048 || P.N == 4096;
  s.cols_block_i = ct_le4096 ? std::min(c.cols_threads, 256) : c.cols_threads;
  s.cols_smem_f = (2 * (size_t)xpad_len(P.N) + kFourStepTw + P.ph_lo + 64) * sizeof(float2);
  s.cols_smem_a = (2 * (size_t)xpad_len(P.N) + kFourStepTw + P.ph_lo + 64) * sizeof(float2);
  s.cols_smem_i = ((size_t)xpad_len(P.N) + kFourStepTw) * sizeof(float2);
  const bool split_ok = split_length(P.N) && P.n <= split_max_rows(P.N);
  s.cols_split_f = split_ok && (c.cols_split & 1);
  s.cols_split_a = split_ok && (c.cols_split & 2);
  s.cols_block_split = 32 * (P.N / 512);
  if (s.cols_split_f) s.cols_smem_f = split_cols_smem(P.N, P.ph_lo + 64);
  if (s.cols_split_a) s.cols_smem_a = split_cols_smem(P.N, P.ph_lo + 64);
  s.ntiles = (P.J + c.rings_per_cta - 1) / c.rings_per_cta;
  s.rings_grid = dim3(s.ntiles + P.n_low, batch);
  s.rings_block = c.rings_per_cta * c.nt_phi;
  s.rings_smem = ((size_t)c.rings_per_cta * xpad_len(P.n_phi) + P.fphi.ptw_len + kFourStepTw) * sizeof(float2) +
                 ((size_t)P.bt_bs + 4) * sizeof(float);  // + the tile's multiplier block, 16-byte aligned
  if (s.rings_smem < 96 * sizeof(float)) s.rings_smem = 96 * sizeof(float);
  s.modes_grid = dim3(P.K + 1, batch);
  s.modes_block = c.nt_2M;
  s.modes_smem = ((size_t)xpad_len(2 * P.M) + P.f2M.ptw_len) * sizeof(float2);
  s.theta_grid = dim3((P.n_t + c.t_tile - 1) / c.t_tile, batch);
  s.theta_block = (c.t_tile / 2) * c.nt_det;
  s.theta_smem = ((size_t)(c.t_tile / 2) * xpad_len(P.n_det) + P.fdet.ptw_len + kFourStepTw) * sizeof(float2);
  return s;
}

template <int V>
using IC = std::integral_constant<int, V>;

// FFT lengths with a compile-time schedule; others use the runtime path.
template <class F>
inline void dispatch_N(int L, F&& f) {
  switch (L) {
    case 256: f(IC<256>{}); break;
    case 512: f(IC<512>{}); break;
    case 1024: f(IC<1024>{}); break;
    case 2048: f(IC<2048>{}); break;
    case 4096: f(IC<4096>{}); break;
    case 8192: f(IC<8192>{}); break;
    default: f(IC<0>{}); break;
  }
}
template <class F>
inline void dispatch_ang(int L, F&& f) {
  switch (L) {
    case 64: f(IC<64>{}); break;
    case 128: f(IC<128>{}); break;
    case 256: f(IC<256>{}); break;
    case 512: f(IC<512>{}); break;
    case 1024: f(IC<1024>{}); break;
    case 2048: f(IC<2048>{}); break;
    case 4096: f(IC<4096>{}); break;
    default: f(IC<0>{}); break;
  }
}
// Pass order of the length-2M transform (compile-time V of the cosine/sine kernels).
template <class F>
inline void dispatch_order(int order, F&& f) {
  if (order == 1) f(IC<1>{});
  else f(IC<0>{});
}
template <class F>
inline void dispatch_2M(int L, F&& f) {
  switch (L) {
    case 384: f(IC<384>{}); break;
    case 768: f(IC<768>{}); break;
    case 1536: f(IC<1536>{}); break;
    case 3072: f(IC<3072>{}); break;
    case 6144: f(IC<6144>{}); break;
    case 12288: f(IC<12288>{}); break;
    default: f(IC<0>{}); break;
  }
}

// Raises the dynamic shared-memory limit of one kernel instantiation once per
// device (cudaFuncSetAttribute is per function and device).
template <auto Kernel>
inline bool ensure_smem(int device) {
  static unsigned long long done = 0;  // one flag set per kernel instantiation
  const unsigned long long bit = 1ull << (device & 63);
  if (done & bit) return true;
  if (cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  done |= bit;
  return true;
}

inline tat_status check_launch(bool attrs_ok) {
  if (!attrs_ok) return TAT_ERR_CUDA;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "tat: kernel launch failed: %s\n", cudaGetErrorString(e));
    return TAT_ERR_CUDA;
  }
  return TAT_OK;
}

}  // namespace
}  // namespace tat
