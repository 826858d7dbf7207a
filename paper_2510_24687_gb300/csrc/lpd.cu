// Kernels of the learned primal-dual reconstruction (Section 4.2.1): the 3x3
// convolution layers of the dual and primal nets with their backward passes,
// the loss and the Adam step.  See include/tat_lpd.h for layouts and
// precision.
//
// The 32 -> 32 layer is an implicit GEMM on the tensor cores: per CTA an
// 8 x 16 pixel tile (one warp per image row of 16 pixels = one m16 tile) and
// K = 9 taps x 32 channels in 18 mma.sync.m16n8k16 steps.  The 10 x 18 x 32
// input halo of each tile arrives by TMA (a 4-D tensor map over the NHWC
// activations, zero fill outside the image, 64-byte swizzle, which keeps the
// fragment loads conflict-free), double-buffered on two mbarriers so that the
// next tile's halo is in flight while the current one's MMAs run; the CTAs are
// persistent and stage the 9 x 32 x 32 weights once, rows padded to 40 BF16.
// Its weight gradient is the GEMM dW[tap] = G'^T In_tap over the pixels, one
// warp per tap, operands fetched with ldmatrix.trans.  The thin layers (2 or 3
// planes -> 32, and 32 -> 1) run on the CUDA cores.
#include <cuda.h>  // CUtensorMap and its enums (types only; the encoder is looked up at run time)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "tat_lpd.h"

namespace {

constexpr int C = 32;       // hidden channels
constexpr int CP = 40;      // padded channel stride in shared memory (BF16 elements)
constexpr int TY = 8, TX = 16;  // output tile of the tensor-core kernels
constexpr int kMaxCtas = 2 * 152;   // CTAs of the tensor-core weight gradient
constexpr int kRedCtas = 8 * 152;   // CTAs of the CUDA-core weight gradients (latency-bound loops)

tat_status launched(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "%s: launch failed: %s\n", what, cudaGetErrorString(e));
    return TAT_ERR_CUDA;
  }
  return TAT_OK;
}

__device__ __forceinline__ float bf(const tat_bf16 v) { return __bfloat162float(__ushort_as_bfloat16(v)); }
__device__ __forceinline__ tat_bf16 tobf(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float rbf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// 8 BF16 values (16 bytes) <-> floats
__device__ __forceinline__ void unpack8(const uint4& u, float* f) {
  const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = bf((tat_bf16)(w[i] & 0xffffu));
    f[2 * i + 1] = bf((tat_bf16)(w[i] >> 16));
  }
}
__device__ __forceinline__ uint4 pack8(const float* f) {
  unsigned w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) w[i] = (unsigned)tobf(f[2 * i]) | ((unsigned)tobf(f[2 * i + 1]) << 16);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

struct Px {
  int b, y, x;
};
__device__ __forceinline__ Px px_of(long long i, int H, int W) {
  Px p;
  const long long hw = (long long)H * W;
  p.b = (int)(i / hw);
  const long long r = i - (long long)p.b * hw;
  p.y = (int)(r / W);
  p.x = (int)(r - (long long)p.y * W);
  return p;
}

#define GRID_STRIDE(i, n) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

int blocks_for(long long n, int threads) {
  const long long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 152LL * 16 ? 152LL * 16 : b));
}

// ------------------------------------------------------------------ in layer (CUDA cores)

template <int CIN>
__global__ void k_conv_in_fwd(int B, int H, int W, const float* __restrict__ x0, const float* __restrict__ x1,
                              const float* __restrict__ x2, const tat_bf16* __restrict__ w,
                              const float* __restrict__ bias, tat_bf16* __restrict__ h) {
  __shared__ float ws[9 * CIN * C];
  __shared__ float bs[C];
  for (int i = threadIdx.x; i < 9 * CIN * C; i += blockDim.x) ws[i] = bf(w[i]);
  for (int i = threadIdx.x; i < C; i += blockDim.x) bs[i] = bias[i];
  __syncthreads();
  const float* xs[3] = {x0, x1, x2};
  const long long hw = (long long)H * W;
  GRID_STRIDE(i, (long long)B * hw) {
    const Px p = px_of(i, H, W);
    float acc[C];
#pragma unroll
    for (int co = 0; co < C; ++co) acc[co] = bs[co];
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = p.y + dy;
      if (yy < 0 || yy >= H) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = p.x + dx;
        if (xx < 0 || xx >= W) continue;
        const int tap = 3 * (dy + 1) + (dx + 1);
        const long long o = (long long)p.b * hw + (long long)yy * W + xx;
#pragma unroll
        for (int c = 0; c < CIN; ++c) {
          const float v = rbf(xs[c][o]);
          const float* wr = ws + (tap * CIN + c) * C;
#pragma unroll
          for (int co = 0; co < C; ++co) acc[co] = fmaf(v, wr[co], acc[co]);
        }
      }
    }
    uint4* dst = reinterpret_cast<uint4*>(h + i * C);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float f[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = fmaxf(acc[8 * q + k], 0.f);
      dst[q] = pack8(f);
    }
  }
}

// G'(pixel) = g_h * [h > 0] as 32 floats
__device__ __forceinline__ void masked_grad(const tat_bf16* g, const tat_bf16* h, long long pix, float* out) {
  const uint4* gp = reinterpret_cast<const uint4*>(g + pix * C);
  const uint4* hp = reinterpret_cast<const uint4*>(h + pix * C);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float gv[8], hv[8];
    unpack8(gp[q], gv);
    unpack8(hp[q], hv);
#pragma unroll
    for (int k = 0; k < 8; ++k) out[8 * q + k] = hv[k] > 0.f ? gv[k] : 0.f;
  }
}

template <int CIN>
__global__ void k_conv_in_bwd_data(int B, int H, int W, const tat_bf16* __restrict__ g_h,
                                   const tat_bf16* __restrict__ h, const tat_bf16* __restrict__ w, float* gx0,
                                   float* gx1, float* gx2, int accumulate) {
  __shared__ float ws[9 * CIN * C];
  for (int i = threadIdx.x; i < 9 * CIN * C; i += blockDim.x) ws[i] = bf(w[i]);
  __syncthreads();
  float* gxs[3] = {gx0, gx1, gx2};
  const long long hw = (long long)H * W;
  GRID_STRIDE(i, (long long)B * hw) {
    const Px p = px_of(i, H, W);
    float acc[CIN];
#pragma unroll
    for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
    // the output pixel (y - dy, x - dx) saw this input through tap (dy, dx)
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = p.y - dy;
      if (yy < 0 || yy >= H) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = p.x - dx;
        if (xx < 0 || xx >= W) continue;
        const int tap = 3 * (dy + 1) + (dx + 1);
        float G[C];
        masked_grad(g_h, h, (long long)p.b * hw + (long long)yy * W + xx, G);
#pragma unroll
        for (int c = 0; c < CIN; ++c) {
          const float* wr = ws + (tap * CIN + c) * C;
          float s = 0.f;
#pragma unroll
          for (int co = 0; co < C; ++co) s = fmaf(G[co], wr[co], s);
          acc[c] += s;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < CIN; ++c)
      if (gxs[c] != nullptr) gxs[c][i] = (((accumulate >> c) & 1) ? gxs[c][i] : 0.f) + acc[c];
  }
}

// Contiguous pixel range [i0, i1) of CTA `blockIdx.x` out of gridDim.x.
__device__ __forceinline__ void cta_range(long long total, long long* i0, long long* i1) {
  const long long per = (total + gridDim.x - 1) / gridDim.x;
  *i0 = (long long)blockIdx.x * per;
  *i1 = *i0 + per < total ? *i0 + per : total;
}

// Per-CTA partial sums of dW[tap][c][co] (9*CIN*C values) and db[co] (C values):
// lane = co, the 8 warps take every 8th pixel of the CTA's range, then the
// warps' sums are added in shared memory.
template <int CIN>
__global__ void __launch_bounds__(256) k_conv_in_bwd_weights(int B, int H, int W, const float* __restrict__ x0,
                                                             const float* __restrict__ x1,
                                                             const float* __restrict__ x2,
                                                             const tat_bf16* __restrict__ g_h,
                                                             const tat_bf16* __restrict__ h, float* partial) {
  constexpr int NW = 9 * CIN * C + C;
  __shared__ float red[8][NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long hw = (long long)H * W;
  long long i0, i1;
  cta_range((long long)B * hw, &i0, &i1);
  float acc[9 * CIN], bacc = 0.f;
#pragma unroll
  for (int k = 0; k < 9 * CIN; ++k) acc[k] = 0.f;
#pragma unroll 4
  for (long long i = i0 + warp; i < i1; i += 8) {
    const float gv = bf(g_h[i * C + lane]), hv = bf(h[i * C + lane]);
    const float G = hv > 0.f ? gv : 0.f;
    bacc += G;
    const Px p = px_of(i, H, W);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = p.y + tap / 3 - 1, xx = p.x + tap % 3 - 1;
      if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
      const long long o = (long long)p.b * hw + (long long)yy * W + xx;
      acc[tap * CIN + 0] = fmaf(G, rbf(x0[o]), acc[tap * CIN + 0]);
      acc[tap * CIN + 1] = fmaf(G, rbf(x1[o]), acc[tap * CIN + 1]);
      if (CIN == 3) acc[tap * CIN + CIN - 1] = fmaf(G, rbf(x2[o]), acc[tap * CIN + CIN - 1]);
    }
  }
#pragma unroll
  for (int k = 0; k < 9 * CIN; ++k) red[warp][k * C + lane] = acc[k];
  red[warp][9 * CIN * C + lane] = bacc;
  __syncthreads();
  for (int o = threadIdx.x; o < NW; o += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w][o];
    partial[(size_t)blockIdx.x * NW + o] = t;
  }
}

// out[e] += sum over CTAs of partial[cta][e] (fixed order); e < nw_w goes to gw[e], the rest to
// gb[e - nw_w].  A block covers 32 outputs (lanes); its 8 warps split the CTAs.
__global__ void __launch_bounds__(256) k_reduce_partials(int nctas, int nw_w, int nb, const float* __restrict__ partial,
                                                         float* gw, float* gb) {
  __shared__ float red[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = nw_w + nb;
  const int e = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (e < nw)
    for (int c = warp; c < nctas; c += 8) s += partial[(size_t)c * nw + e];
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && e < nw) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w][lane];
    if (e < nw_w) gw[e] += t;
    else gb[e - nw_w] += t;
  }
}

// ------------------------------------------------------------------ mid layer (tensor cores)

__device__ __forceinline__ void mma_bf16(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned ld32(const tat_bf16* p) { return *reinterpret_cast<const unsigned*>(p); }

// Loads the (TY+2) x (TX+2) x 32 halo of image b around the tile (y0, x0) into
// hs[(TY+2)*(TX+2)][CP]; out-of-image pixels are zero.  With MASK the value is
// v * [m > 0] (the ReLU mask of the layer's forward output).
template <bool MASK>
__device__ __forceinline__ void load_halo(tat_bf16* hs, const tat_bf16* __restrict__ v, const tat_bf16* __restrict__ m,
                                          int b, int y0, int x0, int H, int W) {
  constexpr int NP = (TY + 2) * (TX + 2);
  for (int e = threadIdx.x; e < NP * 4; e += blockDim.x) {
    const int pix = e >> 2, q = e & 3;
    const int yy = y0 - 1 + pix / (TX + 2), xx = x0 - 1 + pix % (TX + 2);
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
      const long long o = (((long long)b * H + yy) * W + xx) * C + 8 * q;
      u = *reinterpret_cast<const uint4*>(v + o);
      if (MASK) {
        const uint4 mu = *reinterpret_cast<const uint4*>(m + o);
        float fv[8], fm[8];
        unpack8(u, fv);
        unpack8(mu, fm);
#pragma unroll
        for (int k = 0; k < 8; ++k) fv[k] = fm[k] > 0.f ? fv[k] : 0.f;
        u = pack8(fv);
      }
    }
    *reinterpret_cast<uint4*>(hs + pix * CP + 8 * q) = u;
  }
}

// ---- TMA staging of the halo

constexpr int HALO_PIX = (TY + 2) * (TX + 2);  // 180 pixels of 64 bytes
constexpr int HALO_BYTES = HALO_PIX * C * 2;   // 11 520 bytes per tile
constexpr int HALO_SLOT = 12288;               // tile slot, a multiple of the 512-byte swizzle period
constexpr int kSpinLimit = 1 << 22;            // tries of a bounded mbarrier wait before giving up

__device__ int g_lpd_timeout = 0;  // set when a CTA gave up waiting for a tile

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase `parity` of `bar` to complete; false if it did not.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (int i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// One 4-D tile (channels, x, y, image) of `map` into shared memory at `dst`,
// completing `bytes` on `bar`.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// 32-bit word (channels c, c+1) of halo pixel p in a tile written by TMA with
// the 64-byte swizzle: 16-byte chunk j of the 64-byte row p sits at j ^ ((p >> 1) & 3).
__device__ __forceinline__ unsigned ldsw(const unsigned char* tile, int p, int c) {
  const int byte = 2 * c;
  const int chunk = (byte >> 4) ^ ((p >> 1) & 3);
  return *reinterpret_cast<const unsigned*>(tile + p * 64 + (chunk << 4) + (byte & 15));
}

// g * [h > 0] for the two BF16 values of a word (h > 0: sign clear and not zero).
__device__ __forceinline__ unsigned relu_masked(unsigned g, unsigned h) {
  const unsigned lo = h & 0xffffu, hi = h >> 16;
  const unsigned m = ((lo - 1u) < 0x7fffu ? 0x0000ffffu : 0u) | ((hi - 1u) < 0x7fffu ? 0xffff0000u : 0u);
  return g & m;
}

__device__ __forceinline__ void ldsm_x4(unsigned* r, const unsigned char* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

// One 8 x 16 output tile of the mid layer from a staged halo (and, for BWD, the
// staged ReLU mask) and the staged weights.
// FWD: out = relu(conv(in) + b).  BWD (data gradient): out = conv^T(g * [h > 0]),
// i.e. the same implicit GEMM with the taps flipped and in/out channels swapped.
template <bool BWD>
__device__ __forceinline__ void mid_tile(const unsigned char* tile, const unsigned char* mtile, const tat_bf16* wsm,
                                         const float* __restrict__ bias, tat_bf16* __restrict__ out, int b, int y0,
                                         int x0, int H, int W) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[4][4];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[nt][k] = 0.f;
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) {
    const int dy = tap / 3, dx = tap % 3;  // halo offsets (tap - 1 in each direction, plus the halo's +1)
    const int p0 = (warp + dy) * (TX + 2) + g + dx, p1 = p0 + 8;  // pixels g and g + 8 of the warp's row
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
      // A (16 pixels x 16 channels) by one ldmatrix.x4: lane l addresses row l & 7 of
      // matrix l >> 3 = (pixels +8 if odd, channels +8 if >= 2), swizzled 16-byte chunk
      const int m = lane >> 3;
      const int pa = (m & 1 ? p1 : p0) + (lane & 7) - g;
      const int chunk = (2 * kc + (m >> 1)) ^ ((pa >> 1) & 3);
      unsigned a[4];
      ldsm_x4(a, tile + pa * 64 + (chunk << 4));
      if (BWD) {
        unsigned mk[4];
        ldsm_x4(mk, mtile + pa * 64 + (chunk << 4));
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] = relu_masked(a[j], mk[j]);
      }
      // B for n-tiles (2np, 2np+1): matrices (nt 2np, k 0-7), (2np, k 8-15), (2np+1, k 0-7), (2np+1, k 8-15)
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        unsigned bq[4];
        ldsm_x4(bq, reinterpret_cast<const unsigned char*>(
                        wsm + (tap * C + (2 * np + (m >> 1)) * 8 + (lane & 7)) * CP + kc * 16 + (m & 1) * 8));
        mma_bf16(acc[2 * np], a, bq);
        mma_bf16(acc[2 * np + 1], a, bq + 2);
      }
    }
  }
  const int y = y0 + warp;
  if (y >= H) return;  // (no barrier follows inside the tile)
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int x = x0 + g + 8 * half;
    if (x >= W) continue;
    tat_bf16* dst = out + (((long long)b * H + y) * W + x) * C;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int co = nt * 8 + 2 * t;
      float v0 = acc[nt][2 * half], v1 = acc[nt][2 * half + 1];
      if (!BWD) {
        v0 = fmaxf(v0 + bias[co], 0.f);
        v1 = fmaxf(v1 + bias[co + 1], 0.f);
      }
      *reinterpret_cast<unsigned*>(dst + co) = (unsigned)tobf(v0) | ((unsigned)tobf(v1) << 16);
    }
  }
}

// Dynamic shared memory of the mid-layer kernel: alignment slack, two stages
// (value tile, and for BWD the mask tile), the padded weights, two mbarriers.
template <bool BWD>
constexpr size_t mid_smem_bytes() {
  return 1024 + 2 * (BWD ? 2 : 1) * HALO_SLOT + 9 * C * CP * 2 + 2 * sizeof(uint64_t);
}

template <bool BWD>
__global__ void __launch_bounds__(256) k_conv_mid(int B, int H, int W, const __grid_constant__ CUtensorMap map_in,
                                                  const __grid_constant__ CUtensorMap map_mask,
                                                  const tat_bf16* __restrict__ w, const float* __restrict__ bias,
                                                  tat_bf16* __restrict__ out) {
  extern __shared__ unsigned char dsm[];
  unsigned char* sm = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);  // 1024-aligned (swizzle period)
  constexpr int NT = BWD ? 2 : 1;
  constexpr int STAGE = NT * HALO_SLOT;
  tat_bf16* wsm = reinterpret_cast<tat_bf16*>(sm + 2 * STAGE);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * STAGE + 9 * C * CP * 2);
  // weights, read in global order (coalesced): wsm[tap][n][k] with n the output
  // channel of this GEMM and k its input channel
  for (int e = threadIdx.x; e < 9 * C * C; e += blockDim.x) {
    const int tap = e / (C * C), r = e % (C * C), co = r / C, ci = r % C;
    if (BWD) wsm[((8 - tap) * C + ci) * CP + co] = w[e];
    else wsm[(tap * C + co) * CP + ci] = w[e];
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const int tilesx = (W + TX - 1) / TX, tilesy = (H + TY - 1) / TY;
  const long long ntiles = (long long)B * tilesx * tilesy;
  auto coords = [&](long long tile, int* b, int* y0, int* x0) {
    *b = (int)(tile / (tilesx * tilesy));
    const int rr = (int)(tile % (tilesx * tilesy));
    *y0 = (rr / tilesx) * TY;
    *x0 = (rr % tilesx) * TX;
  };
  auto issue = [&](long long tile, int s) {
    if (threadIdx.x != 0) return;
    int b, y0, x0;
    coords(tile, &b, &y0, &x0);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic reads of the slot come first
    mbar_expect_tx(&bar[s], NT * HALO_BYTES);
    tma_load_4d(sm + s * STAGE, &map_in, 0, x0 - 1, y0 - 1, b, &bar[s]);
    if (BWD) tma_load_4d(sm + s * STAGE + HALO_SLOT, &map_mask, 0, x0 - 1, y0 - 1, b, &bar[s]);
  };
  if ((long long)blockIdx.x < ntiles) issue(blockIdx.x, 0);
  int i = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
    const int s = i & 1;
    const long long next = tile + gridDim.x;
    if (next < ntiles) issue(next, s ^ 1);  // that slot was released by the barrier ending the previous tile
    const bool ok = mbar_wait(&bar[s], (unsigned)((i >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      // give up: record it, let the copy still in flight land (bounded), and leave
      if (threadIdx.x == 0) atomicExch(&g_lpd_timeout, 1);
      if (next < ntiles) mbar_wait(&bar[s ^ 1], (unsigned)(((i + 1) >> 1) & 1));
      return;
    }
    int b, y0, x0;
    coords(tile, &b, &y0, &x0);
    mid_tile<BWD>(sm + s * STAGE, sm + s * STAGE + HALO_SLOT, wsm, bias, out, b, y0, x0, H, W);
    __syncthreads();
  }
}

__device__ __forceinline__ void ldsm_x4_trans(unsigned* r, const tat_bf16* p) {
  const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// dW[tap][co][ci] = sum_p G'(p)[co] in(p + tap)[ci], db[co] = sum_p G'(p)[co],
// G' = g * [h_out > 0].  9 warps, warp w = tap w; per-CTA partials.
__global__ void __launch_bounds__(288) k_conv_mid_wgrad(int B, int H, int W, const tat_bf16* __restrict__ in,
                                                        const tat_bf16* __restrict__ g,
                                                        const tat_bf16* __restrict__ hout, float* partial) {
  __shared__ __align__(16) tat_bf16 hs[(TY + 2) * (TX + 2) * CP];
  __shared__ __align__(16) tat_bf16 gs[TY * TX * CP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, t = lane & 3;
  const int tilesx = (W + TX - 1) / TX, tilesy = (H + TY - 1) / TY;
  const long long ntiles = (long long)B * tilesx * tilesy;
  float acc[2][4][4];
#pragma unroll
  for (int mh = 0; mh < 2; ++mh)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[mh][nt][k] = 0.f;
  float bsum = 0.f;  // thread co < 32 of warp 0
  const int dy = warp / 3, dx = warp % 3;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int b = (int)(tile / (tilesx * tilesy));
    const int r = (int)(tile % (tilesx * tilesy));
    const int y0 = (r / tilesx) * TY, x0 = (r % tilesx) * TX;
    __syncthreads();
    load_halo<false>(hs, in, nullptr, b, y0, x0, H, W);
    // masked gradient tile gs[pixel][co], pixel = row * TX + col; zero outside the image
    for (int e = threadIdx.x; e < TY * TX * 4; e += blockDim.x) {
      const int pix = e >> 2, q = e & 3;
      const int yy = y0 + pix / TX, xx = x0 + pix % TX;
      uint4 u = make_uint4(0u, 0u, 0u, 0u);
      if (yy < H && xx < W) {
        const long long o = (((long long)b * H + yy) * W + xx) * C + 8 * q;
        float fv[8], fm[8];
        unpack8(*reinterpret_cast<const uint4*>(g + o), fv);
        unpack8(*reinterpret_cast<const uint4*>(hout + o), fm);
#pragma unroll
        for (int k = 0; k < 8; ++k) fv[k] = fm[k] > 0.f ? fv[k] : 0.f;
        u = pack8(fv);
      }
      *reinterpret_cast<uint4*>(gs + pix * CP + 8 * q) = u;
    }
    __syncthreads();
    if (threadIdx.x < C)
      for (int pix = 0; pix < TY * TX; ++pix) bsum += bf(gs[pix * CP + threadIdx.x]);
    // K loop: one tile row (16 pixels) per step
    const int m = lane >> 3, i = lane & 7;
#pragma unroll 1
    for (int row = 0; row < TY; ++row) {
      unsigned a[2][4];
#pragma unroll
      for (int mh = 0; mh < 2; ++mh) {
        // matrices: (co 0-7, px 0-7), (co 8-15, px 0-7), (co 0-7, px 8-15), (co 8-15, px 8-15) of A = G'^T
        const int px = (m >= 2 ? 8 : 0) + i, co = mh * 16 + ((m & 1) ? 8 : 0);
        ldsm_x4_trans(a[mh], gs + (row * TX + px) * CP + co);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        // matrices: (ci of n-tile 2np, px 0-7), (2np, px 8-15), (2np+1, px 0-7), (2np+1, px 8-15)
        const int px = ((m & 1) ? 8 : 0) + i, ci = (2 * np + (m >> 1)) * 8;
        unsigned bq[4];
        ldsm_x4_trans(bq, hs + ((row + dy) * (TX + 2) + px + dx) * CP + ci);
#pragma unroll
        for (int mh = 0; mh < 2; ++mh) {
          mma_bf16(acc[mh][2 * np], a[mh], bq);
          mma_bf16(acc[mh][2 * np + 1], a[mh], bq + 2);
        }
      }
    }
  }
  // partial layout: [tap][co][ci] then [co] for the bias
  constexpr int NW = 9 * C * C + C;
  float* pp = partial + (size_t)blockIdx.x * NW;
#pragma unroll
  for (int mh = 0; mh < 2; ++mh)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int co = mh * 16 + gq, ci = nt * 8 + 2 * t;
      float* d0 = pp + (warp * C + co) * C + ci;
      float* d1 = pp + (warp * C + co + 8) * C + ci;
      d0[0] = acc[mh][nt][0];
      d0[1] = acc[mh][nt][1];
      d1[0] = acc[mh][nt][2];
      d1[1] = acc[mh][nt][3];
    }
  if (threadIdx.x < C) pp[9 * C * C + threadIdx.x] = bsum;
}

// ------------------------------------------------------------------ out layer (CUDA cores)

__global__ void k_conv_out_fwd(int B, int H, int W, const tat_bf16* __restrict__ h, const tat_bf16* __restrict__ w,
                               const float* __restrict__ bias, const float* residual, float* out) {
  __shared__ float ws[9 * C];
  for (int i = threadIdx.x; i < 9 * C; i += blockDim.x) ws[i] = bf(w[i]);
  __syncthreads();
  const long long hw = (long long)H * W;
  const float b0 = bias[0];
  GRID_STRIDE(i, (long long)B * hw) {
    const Px p = px_of(i, H, W);
    float acc = b0;
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = p.y + dy;
      if (yy < 0 || yy >= H) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = p.x + dx;
        if (xx < 0 || xx >= W) continue;
        const float* wr = ws + (3 * (dy + 1) + (dx + 1)) * C;
        const uint4* src = reinterpret_cast<const uint4*>(h + ((long long)p.b * hw + (long long)yy * W + xx) * C);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float f[8];
          unpack8(src[q], f);
#pragma unroll
          for (int k = 0; k < 8; ++k) acc = fmaf(f[k], wr[8 * q + k], acc);
        }
      }
    }
    out[i] = residual[i] + acc;
  }
}

__global__ void k_conv_out_bwd_data(int B, int H, int W, const float* __restrict__ gout,
                                    const tat_bf16* __restrict__ w, tat_bf16* __restrict__ gh) {
  __shared__ float ws[9 * C];
  for (int i = threadIdx.x; i < 9 * C; i += blockDim.x) ws[i] = bf(w[i]);
  __syncthreads();
  const long long hw = (long long)H * W;
  GRID_STRIDE(i, (long long)B * hw) {
    const Px p = px_of(i, H, W);
    float acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0.f;
    for (int dy = -1; dy <= 1; ++dy) {
      const int yy = p.y - dy;
      if (yy < 0 || yy >= H) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = p.x - dx;
        if (xx < 0 || xx >= W) continue;
        const float gv = gout[(long long)p.b * hw + (long long)yy * W + xx];
        const float* wr = ws + (3 * (dy + 1) + (dx + 1)) * C;
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = fmaf(gv, wr[c], acc[c]);
      }
    }
    uint4* dst = reinterpret_cast<uint4*>(gh + i * C);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[q] = pack8(acc + 8 * q);
  }
}

// Per-CTA partials of dW[tap][ci] (288) and db (1): lane = ci, the 8 warps take
// every 8th pixel of the CTA's range, then the warps' sums are added in shared memory.
__global__ void __launch_bounds__(256) k_conv_out_wgrad(int B, int H, int W, const float* __restrict__ gout,
                                                        const tat_bf16* __restrict__ h, float* partial) {
  constexpr int NW = 9 * C + 1;
  __shared__ float red[8][NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long hw = (long long)H * W;
  long long i0, i1;
  cta_range((long long)B * hw, &i0, &i1);
  float acc[9], bacc = 0.f;
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.f;
#pragma unroll 4
  for (long long i = i0 + warp; i < i1; i += 8) {
    const float gv = gout[i];
    bacc += gv;
    const Px p = px_of(i, H, W);
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int yy = p.y + tap / 3 - 1, xx = p.x + tap % 3 - 1;
      if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
      acc[tap] = fmaf(gv, bf(h[((long long)p.b * hw + (long long)yy * W + xx) * C + lane]), acc[tap]);
    }
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) red[warp][k * C + lane] = acc[k];
  if (lane == 0) red[warp][9 * C] = bacc;
  __syncthreads();
  for (int o = threadIdx.x; o < NW; o += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w][o];
    partial[(size_t)blockIdx.x * NW + o] = t;
  }
}

// ------------------------------------------------------------------ optimizer and loss

__global__ void k_adam(long long n, float lr, float b1, float b2, float eps, float c1, float c2, float* p,
                       const float* __restrict__ g, float* m, float* v, tat_bf16* wb) {
  GRID_STRIDE(i, n) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (wb != nullptr) wb[i] = tobf(pi);
  }
}

__global__ void k_fill(long long n, float value, float* out) {
  GRID_STRIDE(i, n) out[i] = value;
}

__global__ void k_to_bf16(long long n, const float* __restrict__ x, tat_bf16* out) {
  GRID_STRIDE(i, n) out[i] = tobf(x[i]);
}

__global__ void k_mse(long long n, const float* __restrict__ a, const float* __restrict__ b, float scale, float* grad,
                      float* loss) {
  float s = 0.f;
  GRID_STRIDE(i, n) {
    const float d = a[i] - b[i];
    if (grad != nullptr) grad[i] = 2.f * scale * d;
    s = fmaf(d, d, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tsum = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tsum += red[k];
    atomicAdd(loss, scale * tsum);
  }
}

bool bad_sizes(int batch, int H, int W) { return batch < 1 || H < 1 || W < 1; }

// Persistent tensor-core conv: up to 3 CTAs per SM, every CTA stages the
// weights once and loops over tiles.
int mid_ctas(int batch, int H, int W) {
  const long long tiles = (long long)batch * ((H + TY - 1) / TY) * ((W + TX - 1) / TX);
  return (int)(tiles < 3 * 152 ? tiles : 3 * 152);
}

// cuTensorMapEncodeTiled, looked up through the runtime (no link-time driver dependency).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of a [batch][H][W][32] BF16 activation for (TY+2) x (TX+2) x 32 halo boxes.
bool halo_map(CUtensorMap* m, const tat_bf16* base, int batch, int H, int W) {
  const EncodeTiled fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)batch};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
  const cuuint32_t box[4] = {(cuuint32_t)C, TX + 2, TY + 2, 1};
  const cuuint32_t estride[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<tat_bf16*>(base), dims, strides, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool BWD>
tat_status launch_mid(int batch, int H, int W, const tat_bf16* in, const tat_bf16* mask, const tat_bf16* w,
                      const float* b, tat_bf16* out, cudaStream_t s, const char* what) {
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(mask)) & 15) return TAT_ERR_INVALID_ARG;
  CUtensorMap mi, mm;
  if (!halo_map(&mi, in, batch, H, W) || !halo_map(&mm, BWD ? mask : in, batch, H, W)) {
    fprintf(stderr, "%s: tensor map encoding failed\n", what);
    return TAT_ERR_CUDA;
  }
  static int attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    if (cudaFuncSetAttribute(k_conv_mid<BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)mid_smem_bytes<BWD>()) != cudaSuccess) {
      cudaGetLastError();
      return TAT_ERR_CUDA;
    }
    attr_done[dev] = 1;
  }
  k_conv_mid<BWD><<<mid_ctas(batch, H, W), 256, mid_smem_bytes<BWD>(), s>>>(batch, H, W, mi, mm, w, b, out);
  return launched(what);
}

int wgrad_ctas(int batch, int H, int W) {
  const long long tiles = (long long)batch * ((H + TY - 1) / TY) * ((W + TX - 1) / TX);
  return (int)(tiles < kMaxCtas ? tiles : kMaxCtas);
}

}  // namespace

extern "C" {

size_t tat_lpd_scratch_floats(int batch, int H, int W) {
  if (bad_sizes(batch, H, W)) return 0;
  const size_t a = (size_t)kMaxCtas * (9 * C * C + C), b = (size_t)kRedCtas * (9 * 3 * C + C);
  return a > b ? a : b;
}

tat_status tat_conv_in_fwd(int batch, int H, int W, int cin, const float* x0, const float* x1, const float* x2,
                           const tat_bf16* w, const float* b, tat_bf16* h, tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || (cin != 2 && cin != 3) || !x0 || !x1 || (cin == 3 && !x2) || !w || !b || !h)
    return TAT_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long n = (long long)batch * H * W;
  if (cin == 2) k_conv_in_fwd<2><<<blocks_for(n, 256), 256, 0, s>>>(batch, H, W, x0, x1, nullptr, w, b, h);
  else k_conv_in_fwd<3><<<blocks_for(n, 256), 256, 0, s>>>(batch, H, W, x0, x1, x2, w, b, h);
  return launched("tat_conv_in_fwd");
}

tat_status tat_conv_in_bwd_data(int batch, int H, int W, int cin, const tat_bf16* g_h, const tat_bf16* h,
                                const tat_bf16* w, float* gx0, float* gx1, float* gx2, int accumulate,
                                tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || (cin != 2 && cin != 3) || !g_h || !h || !w) return TAT_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long n = (long long)batch * H * W;
  if (cin == 2) k_conv_in_bwd_data<2><<<blocks_for(n, 256), 256, 0, s>>>(batch, H, W, g_h, h, w, gx0, gx1, nullptr, accumulate);
  else k_conv_in_bwd_data<3><<<blocks_for(n, 256), 256, 0, s>>>(batch, H, W, g_h, h, w, gx0, gx1, gx2, accumulate);
  return launched("tat_conv_in_bwd_data");
}

tat_status tat_conv_in_bwd_weights(int batch, int H, int W, int cin, const float* x0, const float* x1,
                                   const float* x2, const tat_bf16* g_h, const tat_bf16* h, float* scratch,
                                   size_t scratch_floats, float* gw, float* gb, tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || (cin != 2 && cin != 3) || !x0 || !x1 || (cin == 3 && !x2) || !g_h || !h ||
      !scratch || !gw || !gb)
    return TAT_ERR_INVALID_ARG;
  const int nw = 9 * cin * C + C;
  const long long total = (long long)batch * H * W;
  const int ctas = (int)((total + 63) / 64 < kRedCtas ? (total + 63) / 64 : kRedCtas);
  if (scratch_floats < (size_t)ctas * nw) return TAT_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cin == 2) k_conv_in_bwd_weights<2><<<ctas, 256, 0, s>>>(batch, H, W, x0, x1, nullptr, g_h, h, scratch);
  else k_conv_in_bwd_weights<3><<<ctas, 256, 0, s>>>(batch, H, W, x0, x1, x2, g_h, h, scratch);
  tat_status st = launched("tat_conv_in_bwd_weights");
  if (st != TAT_OK) return st;
  k_reduce_partials<<<(nw + 31) / 32, 256, 0, s>>>(ctas, 9 * cin * C, C, scratch, gw, gb);
  return launched("tat_conv_in_bwd_weights");
}

tat_status tat_conv_mid_fwd(int batch, int H, int W, const tat_bf16* h_in, const tat_bf16* w, const float* b,
                            tat_bf16* h_out, tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || !h_in || !w || !b || !h_out) return TAT_ERR_INVALID_ARG;
  return launch_mid<false>(batch, H, W, h_in, nullptr, w, b, h_out, static_cast<cudaStream_t>(stream),
                           "tat_conv_mid_fwd");
}

tat_status tat_conv_mid_bwd_data(int batch, int H, int W, const tat_bf16* g_out, const tat_bf16* h_out,
                                 const tat_bf16* w, tat_bf16* g_in, tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || !g_out || !h_out || !w || !g_in) return TAT_ERR_INVALID_ARG;
  return launch_mid<true>(batch, H, W, g_out, h_out, w, nullptr, g_in, static_cast<cudaStream_t>(stream),
                          "tat_conv_mid_bwd_data");
}

tat_status tat_lpd_check(void) {
  int flag = 0;
  if (cudaMemcpyFromSymbol(&flag, g_lpd_timeout, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return TAT_ERR_CUDA;
  }
  if (!flag) return TAT_OK;
  const int zero = 0;
  cudaMemcpyToSymbol(g_lpd_timeout, &zero, sizeof(int));
  return TAT_ERR_TIMEOUT;
}

tat_status tat_conv_mid_bwd_weights(int batch, int H, int W, const tat_bf16* h_in, const tat_bf16* g_out,
                                    const tat_bf16* h_out, float* scratch, size_t scratch_floats, float* gw,
                                    float* gb, tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || !h_in || !g_out || !h_out || !scratch || !gw || !gb) return TAT_ERR_INVALID_ARG;
  const int ctas = wgrad_ctas(batch, H, W);
  const int nw = 9 * C * C + C;
  if (scratch_floats < (size_t)ctas * nw) return TAT_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_conv_mid_wgrad<<<ctas, 288, 0, s>>>(batch, H, W, h_in, g_out, h_out, scratch);
  tat_status st = launched("tat_conv_mid_bwd_weights");
  if (st != TAT_OK) return st;
  k_reduce_partials<<<(nw + 31) / 32, 256, 0, s>>>(ctas, 9 * C * C, C, scratch, gw, gb);
  return launched("tat_conv_mid_bwd_weights");
}

tat_status tat_conv_out_fwd(int batch, int H, int W, const tat_bf16* h, const tat_bf16* w, const float* b,
                            const float* residual, float* out, tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || !h || !w || !b || !residual || !out) return TAT_ERR_INVALID_ARG;
  const long long n = (long long)batch * H * W;
  k_conv_out_fwd<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(batch, H, W, h, w, b, residual,
                                                                                      out);
  return launched("tat_conv_out_fwd");
}

tat_status tat_conv_out_bwd(int batch, int H, int W, const float* g_out, const tat_bf16* h, const tat_bf16* w,
                            tat_bf16* g_h, float* scratch, size_t scratch_floats, float* gw, float* gb,
                            tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || !g_out || !h || !w || !g_h || !scratch || !gw || !gb) return TAT_ERR_INVALID_ARG;
  const long long n = (long long)batch * H * W;
  const int ctas = (int)((n + 63) / 64 < kRedCtas ? (n + 63) / 64 : kRedCtas);
  if (scratch_floats < (size_t)ctas * (9 * C + 1)) return TAT_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_conv_out_bwd_data<<<blocks_for(n, 256), 256, 0, s>>>(batch, H, W, g_out, w, g_h);
  tat_status st = launched("tat_conv_out_bwd");
  if (st != TAT_OK) return st;
  k_conv_out_wgrad<<<ctas, 256, 0, s>>>(batch, H, W, g_out, h, scratch);
  st = launched("tat_conv_out_bwd");
  if (st != TAT_OK) return st;
  k_reduce_partials<<<(9 * C + 1 + 31) / 32, 256, 0, s>>>(ctas, 9 * C, 1, scratch, gw, gb);
  return launched("tat_conv_out_bwd");
}

tat_status tat_adam(long long count, float lr, float beta1, float beta2, float eps, int step, float* param,
                    const float* grad, float* m, float* v, tat_bf16* w_bf16, tat_stream_t stream) {
  if (count <= 0 || step < 1 || !param || !grad || !m || !v) return TAT_ERR_INVALID_ARG;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<blocks_for(count, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(count, lr, beta1, beta2, eps, c1, c2,
                                                                                 param, grad, m, v, w_bf16);
  return launched("tat_adam");
}

tat_status tat_fill(long long count, float value, float* out, tat_stream_t stream) {
  if (count <= 0 || !out) return TAT_ERR_INVALID_ARG;
  k_fill<<<blocks_for(count, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(count, value, out);
  return launched("tat_fill");
}

tat_status tat_to_bf16(long long count, const float* x, tat_bf16* out, tat_stream_t stream) {
  if (count <= 0 || !x || !out) return TAT_ERR_INVALID_ARG;
  k_to_bf16<<<blocks_for(count, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(count, x, out);
  return launched("tat_to_bf16");
}

tat_status tat_mse(long long count, const float* a, const float* b, float scale, float* grad, float* loss,
                   tat_stream_t stream) {
  if (count <= 0 || !a || !b || !loss) return TAT_ERR_INVALID_ARG;
  k_mse<<<blocks_for(count, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(count, a, b, scale, grad, loss);
  return launched("tat_mse");
}

}  // extern "C"
