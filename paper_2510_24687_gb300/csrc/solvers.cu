// Fused element-wise steps of the NNLS and TV-PDHG solvers of Section 4.2
// and their backward passes.  The operator applications themselves are
// tat_forward / tat_adjoint; the update formulas are stated in
// include/tat_solvers.h.
//
// All kernels are grid-stride loops over pixels (or samples) with coalesced
// float loads: they are HBM-bound, so the grid is a fixed multiple of the SM
// count and every array is touched once per call (neighbour reads of the
// gradient stencils hit L1/L2).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "pdl.cuh"
#include "tat_solvers.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 152 * 8;

int blocks_for(long long count) {
  const long long b = (count + kThreads - 1) / kThreads;
  return (int)(b < 1 ? 1 : (b > kMaxBlocks ? kMaxBlocks : b));
}

tat_status launched(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "%s: launch failed: %s\n", what, cudaGetErrorString(e));
    return TAT_ERR_CUDA;
  }
  return TAT_OK;
}

#define TAT_GRID_STRIDE(i, count)                                                  \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (count); \
       i += (long long)gridDim.x * blockDim.x)

// Forward difference of plane `v` at pixel r = iy*n + ix, divided by h
// (zero across the last column / row).
__device__ __forceinline__ float diff_x(const float* v, long long r, int ix, int n, float ih) {
  return ix < n - 1 ? (v[r + 1] - v[r]) * ih : 0.f;
}
__device__ __forceinline__ float diff_y(const float* v, long long r, int iy, int n, float ih) {
  return iy < n - 1 ? (v[r + n] - v[r]) * ih : 0.f;
}

// div_h = -grad_h^T of the field (px, py) at pixel r.
__device__ __forceinline__ float div_at(const float* px, const float* py, long long r, int ix, int iy, int n,
                                        float ih) {
  const float dx = (ix < n - 1 ? px[r] : 0.f) - (ix > 0 ? px[r - 1] : 0.f);
  const float dy = (iy < n - 1 ? py[r] : 0.f) - (iy > 0 ? py[r - n] : 0.f);
  return (dx + dy) * ih;
}

__global__ void k_axpby_clamp(long long count, float a, const float* __restrict__ x, float b,
                              const float* __restrict__ y, float lo, const float* __restrict__ mask,
                              long long period, float* out) {
  TAT_GRID_DEPENDENCY();
  TAT_GRID_STRIDE(i, count) {
    float v = a * x[i];
    if (y != nullptr) v += b * y[i];
    v = fmaxf(v, lo);
    if (mask != nullptr) v *= mask[i % period];
    out[i] = v;
  }
}

__global__ void k_axpby_clamp_backward(long long count, const float* __restrict__ out, float lo,
                                       const float* __restrict__ mask, long long period,
                                       const float* __restrict__ go, float a, float* gx, float b, float* gy) {
  TAT_GRID_DEPENDENCY();
  TAT_GRID_STRIDE(i, count) {
    float G = out[i] > lo ? go[i] : 0.f;
    if (mask != nullptr) G *= mask[i % period];
    if (gx != nullptr) gx[i] = a * G;
    if (gy != nullptr) gy[i] = b * G;
  }
}

__global__ void k_pd_dual_data(long long count, float sigma, float inv, const float* __restrict__ Af,
                               const float* __restrict__ g, const float* q_in, float* q_out) {
  TAT_GRID_DEPENDENCY();
  TAT_GRID_STRIDE(i, count) { q_out[i] = (q_in[i] + sigma * (Af[i] - g[i])) * inv; }
}

struct Pix {
  long long b, r;
  int ix, iy;
};

__device__ __forceinline__ Pix pixel(long long i, int n, long long nn) {
  Pix P;
  P.b = i / nn;
  P.r = i - P.b * nn;
  P.iy = (int)(P.r / n);
  P.ix = (int)(P.r - (long long)P.iy * n);
  return P;
}

__global__ void k_tv_dual(int batch, int n, float ih, float sigma, float bound, const float* __restrict__ fbar,
                          const float* p_in, float* p_out) {
  TAT_GRID_DEPENDENCY();
  const long long nn = (long long)n * n;
  TAT_GRID_STRIDE(i, nn * batch) {
    const Pix P = pixel(i, n, nn);
    const float* fb = fbar + P.b * nn;
    const long long o = 2 * P.b * nn + P.r;
    const float ux = p_in[o] + sigma * diff_x(fb, P.r, P.ix, n, ih);
    const float uy = p_in[o + nn] + sigma * diff_y(fb, P.r, P.iy, n, ih);
    const float s = fmaxf(1.f, sqrtf(ux * ux + uy * uy) / bound);
    p_out[o] = ux / s;
    p_out[o + nn] = uy / s;
  }
}

// grad_p_in = DP(u)^T grad_p_out, with u recomputed from p_in and fbar.
__global__ void k_tv_dual_backward(int batch, int n, float ih, float sigma, float bound,
                                   const float* __restrict__ fbar, const float* __restrict__ p_in,
                                   const float* __restrict__ go, float* gp) {
  TAT_GRID_DEPENDENCY();
  const long long nn = (long long)n * n;
  TAT_GRID_STRIDE(i, nn * batch) {
    const Pix P = pixel(i, n, nn);
    const float* fb = fbar + P.b * nn;
    const long long o = 2 * P.b * nn + P.r;
    const float ux = p_in[o] + sigma * diff_x(fb, P.r, P.ix, n, ih);
    const float uy = p_in[o + nn] + sigma * diff_y(fb, P.r, P.iy, n, ih);
    const float gx = go[o], gy = go[o + nn];
    const float nrm = sqrtf(ux * ux + uy * uy);
    if (nrm <= bound) {
      gp[o] = gx;
      gp[o + nn] = gy;
    } else {
      // (bound/|u|) (I - u u^T / |u|^2) is symmetric.
      const float c = bound / nrm;
      const float dot = (ux * gx + uy * gy) / (nrm * nrm);
      gp[o] = c * (gx - ux * dot);
      gp[o + nn] = c * (gy - uy * dot);
    }
  }
}

// out = scale * div_h(field) per image (the grad_h^T half of the dual backward).
__global__ void k_scaled_div(int batch, int n, float ih, float scale, const float* __restrict__ field, float* out) {
  TAT_GRID_DEPENDENCY();
  const long long nn = (long long)n * n;
  TAT_GRID_STRIDE(i, nn * batch) {
    const Pix P = pixel(i, n, nn);
    const float* px = field + 2 * P.b * nn;
    out[i] = scale * div_at(px, px + nn, P.r, P.ix, P.iy, n, ih);
  }
}

__global__ void k_tv_primal(int batch, int n, float ih, float tau, const float* __restrict__ Asq,
                            const float* __restrict__ p, const float* __restrict__ mask, const float* f_in,
                            float* f_out, float* fbar) {
  TAT_GRID_DEPENDENCY();
  const long long nn = (long long)n * n;
  TAT_GRID_STRIDE(i, nn * batch) {
    const Pix P = pixel(i, n, nn);
    const float* px = p + 2 * P.b * nn;
    const float div = div_at(px, px + nn, P.r, P.ix, P.iy, n, ih);
    const float f0 = f_in[i];
    float fn = fmaxf(0.f, f0 - tau * (Asq[i] - div));
    if (mask != nullptr) fn *= mask[P.r];
    f_out[i] = fn;
    fbar[i] = 2.f * fn - f0;
  }
}

// D of the primal backward at flat index i (pixel r of its image).
__device__ __forceinline__ float primal_D(const float* f_out, const float* mask, const float* gfo, const float* gfb,
                                          long long i, long long r) {
  float G = 0.f;
  if (gfo != nullptr) G += gfo[i];
  if (gfb != nullptr) G += 2.f * gfb[i];
  G = f_out[i] > 0.f ? G : 0.f;
  if (mask != nullptr) G *= mask[r];
  return G;
}

__global__ void k_tv_primal_backward(int batch, int n, float ih, float tau, const float* __restrict__ f_out,
                                     const float* __restrict__ mask, const float* __restrict__ gfo,
                                     const float* __restrict__ gfb, float* gf, float* gA, float* gp) {
  TAT_GRID_DEPENDENCY();
  const long long nn = (long long)n * n;
  TAT_GRID_STRIDE(i, nn * batch) {
    const Pix P = pixel(i, n, nn);
    const float D = primal_D(f_out, mask, gfo, gfb, i, P.r);
    if (gf != nullptr) gf[i] = D - (gfb != nullptr ? gfb[i] : 0.f);
    if (gA != nullptr) gA[i] = -tau * D;
    if (gp != nullptr) {
      const float Dx = P.ix < n - 1 ? primal_D(f_out, mask, gfo, gfb, i + 1, P.r + 1) : D;
      const float Dy = P.iy < n - 1 ? primal_D(f_out, mask, gfo, gfb, i + n, P.r + n) : D;
      const long long o = 2 * P.b * nn + P.r;
      gp[o] = -tau * (Dx - D) * ih;
      gp[o + nn] = -tau * (Dy - D) * ih;
    }
  }
}

bool bad_image_args(int batch, int n, float h_eff) { return batch < 1 || n < 2 || !(h_eff > 0.f); }

}  // namespace

extern "C" {

tat_status tat_axpby_clamp(long long count, float a, const float* x, float b, const float* y, float lo,
                           const float* mask, long long mask_period, float* out, tat_stream_t stream) {
  if (count <= 0 || !x || !out || (mask && mask_period <= 0)) return TAT_ERR_INVALID_ARG;
  tat::pdl_launch(true, k_axpby_clamp, blocks_for(count), kThreads, 0, static_cast<cudaStream_t>(stream), count, a, x, b, y, lo, mask, mask ? mask_period : 1, out);
  return launched("tat_axpby_clamp");
}

tat_status tat_axpby_clamp_backward(long long count, const float* out, float lo, const float* mask,
                                    long long mask_period, const float* grad_out, float a, float* grad_x, float b,
                                    float* grad_y, tat_stream_t stream) {
  if (count <= 0 || !out || !grad_out || (mask && mask_period <= 0)) return TAT_ERR_INVALID_ARG;
  if (!grad_x && !grad_y) return TAT_OK;
  tat::pdl_launch(true, k_axpby_clamp_backward, blocks_for(count), kThreads, 0, static_cast<cudaStream_t>(stream), count, out, lo, mask, mask ? mask_period : 1, grad_out, a, grad_x, b, grad_y);
  return launched("tat_axpby_clamp_backward");
}

tat_status tat_pd_dual_data(long long count, float sigma, const float* Af, const float* g, const float* q_in,
                            float* q_out, tat_stream_t stream) {
  if (count <= 0 || !Af || !g || !q_in || !q_out || !(sigma > 0.f)) return TAT_ERR_INVALID_ARG;
  tat::pdl_launch(true, k_pd_dual_data, blocks_for(count), kThreads, 0, static_cast<cudaStream_t>(stream), count, sigma, 1.f / (1.f + sigma), Af, g, q_in, q_out);
  return launched("tat_pd_dual_data");
}

tat_status tat_tv_dual(int batch, int n, float h_eff, float sigma, float bound, const float* fbar, const float* p_in,
                       float* p_out, tat_stream_t stream) {
  if (bad_image_args(batch, n, h_eff) || !(sigma > 0.f) || !(bound > 0.f) || !fbar || !p_in || !p_out)
    return TAT_ERR_INVALID_ARG;
  const long long count = (long long)batch * n * n;
  tat::pdl_launch(true, k_tv_dual, blocks_for(count), kThreads, 0, static_cast<cudaStream_t>(stream), batch, n, 1.f / h_eff, sigma, bound, fbar, p_in, p_out);
  return launched("tat_tv_dual");
}

tat_status tat_tv_dual_backward(int batch, int n, float h_eff, float sigma, float bound, const float* fbar,
                                const float* p_in, const float* grad_p_out, float* grad_p_in, float* grad_fbar,
                                tat_stream_t stream) {
  if (bad_image_args(batch, n, h_eff) || !(sigma > 0.f) || !(bound > 0.f) || !fbar || !p_in || !grad_p_out ||
      !grad_p_in)
    return TAT_ERR_INVALID_ARG;
  const long long count = (long long)batch * n * n;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  tat::pdl_launch(true, k_tv_dual_backward, blocks_for(count), kThreads, 0, s, batch, n, 1.f / h_eff, sigma, bound, fbar, p_in, grad_p_out, grad_p_in);
  const tat_status st = launched("tat_tv_dual_backward");
  if (st != TAT_OK || !grad_fbar) return st;
  tat::pdl_launch(true, k_scaled_div, blocks_for(count), kThreads, 0, s, batch, n, 1.f / h_eff, -sigma, grad_p_in, grad_fbar);
  return launched("tat_tv_dual_backward");
}

tat_status tat_tv_primal(int batch, int n, float h_eff, float tau, const float* Asq, const float* p, const float* mask,
                         const float* f_in, float* f_out, float* fbar, tat_stream_t stream) {
  if (bad_image_args(batch, n, h_eff) || !(tau > 0.f) || !Asq || !p || !f_in || !f_out || !fbar)
    return TAT_ERR_INVALID_ARG;
  const long long count = (long long)batch * n * n;
  tat::pdl_launch(true, k_tv_primal, blocks_for(count), kThreads, 0, static_cast<cudaStream_t>(stream), batch, n, 1.f / h_eff, tau, Asq, p, mask, f_in, f_out, fbar);
  return launched("tat_tv_primal");
}

tat_status tat_tv_primal_backward(int batch, int n, float h_eff, float tau, const float* f_out, const float* mask,
                                  const float* grad_f_out, const float* grad_fbar, float* grad_f_in, float* grad_Asq,
                                  float* grad_p, tat_stream_t stream) {
  if (bad_image_args(batch, n, h_eff) || !(tau > 0.f) || !f_out) return TAT_ERR_INVALID_ARG;
  const long long count = (long long)batch * n * n;
  tat::pdl_launch(true, k_tv_primal_backward, blocks_for(count), kThreads, 0, static_cast<cudaStream_t>(stream), batch, n, 1.f / h_eff, tau, f_out, mask, grad_f_out, grad_fbar, grad_f_in, grad_Asq, grad_p);
  return launched("tat_tv_primal_backward");
}

}  // extern "C"
