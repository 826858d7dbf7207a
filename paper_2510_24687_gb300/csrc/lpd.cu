// Kernels of the learned primal-dual reconstruction (Section 4.2.1): the 3x3
// convolution layers of the dual and primal nets with their backward passes,
// the loss and the Adam step.  See include/tat_lpd.h for layouts and
// precision.
//
// The 32 -> 32 layer runs on the 5th-generation tensor cores (tcgen05, accumulators in
// TMEM): the forward and the data gradient of an already masked gradient as an implicit
// GEMM per 16 x 8-pixel tile (k_conv_mid_tc), the weight gradient of an already masked
// gradient with four pixel-shifted copies of G' stacked in M (k_conv_mid_wgrad_tc).  The
// variants that read the gradient's ReLU mask themselves run on mma.sync m16n8k16
// (k_conv_mid, k_conv_mid_wgrad): per CTA an 8 x 16 pixel tile, one warp per image row of
// 16 pixels, K = 9 taps x 32 channels in 18 steps.  Every halo arrives by TMA (4-D tensor
// maps over the NHWC activations, zero fill outside the image, 64-byte swizzle); the CTAs
// are persistent.  The thin layers (2 or 3 planes -> 32, and 32 -> 1) are implicit GEMMs
// on mma.sync with one dimension of 8 to 27 -- the 32 -> 1 forward and the in layer's data
// gradient as per-tap channel sums of each halo pixel followed by a 9-point stencil -- and
// their backward passes compute the data and the weight gradients in one pass over the
// tiles.  Weight gradients leave per-CTA partial sums that k_reduce_partials adds in a
// fixed order.
#include <cuda.h>  // CUtensorMap and its enums (types only; the encoder is looked up at run time)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "pdl.cuh"
#include "tat_lpd.h"

namespace {

constexpr int C = 32;       // hidden channels
constexpr int CP = 40;      // padded channel stride in shared memory (BF16 elements)
constexpr int TY = 8, TX = 16;  // output tile of the tensor-core kernels
constexpr int kMaxCtas = 2 * 152;   // CTAs of the 32 -> 32 weight gradient
constexpr int XH = TY + 2, XW = TX + 2;  // 10 x 18 halo of a tile
constexpr int XP = 20;              // row pitch (BF16 elements) of the halo copies of FP32 planes

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

#define GRID_STRIDE(i, n) \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

int blocks_for(long long n, int threads) {
  const long long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > 152LL * 16 ? 152LL * 16 : b));
}

// ------------------------------------------------------------------ weight-gradient partial sums

// out[e] += sum over CTAs of partial[cta][e] (fixed order); e < nw_w goes to gw[e], the rest to
// gb[e - nw_w].  A block covers 32 outputs (lanes); its 32 warps split the CTAs, so that each
// warp adds about ten partials (the sums are short, latency-bound chains otherwise).
__global__ void __launch_bounds__(1024) k_reduce_partials(int nctas, int nw_w, int nb, const float* __restrict__ partial,
                                                          float* gw, float* gb) {
  TAT_GRID_DEPENDENCY();
  __shared__ float red[32][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = nw_w + nb;
  const int e = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (e < nw) {
#pragma unroll 4
    for (int c = warp; c < nctas; c += 32) s += partial[(size_t)c * nw + e];
  }
  red[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && e < nw) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < 32; ++w) t += red[w][lane];
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


// ---- TMA staging of the halo

constexpr int HALO_PIX = (TY + 2) * (TX + 2);  // 180 pixels of 64 bytes
constexpr int HALO_BYTES = HALO_PIX * C * 2;   // 11 520 bytes per tile
constexpr int HALO_SLOT = 12288;               // tile slot, a multiple of the 512-byte swizzle period
constexpr int ZP = 196;  // pitch of per-tap sums over a halo: 192 rows (12 m-tiles) + 4, so that fragment
                         // stores spread over all banks
constexpr int kSpinLimit = 1 << 22;            // tries of a bounded mbarrier wait before giving up

__device__ int g_lpd_timeout = 0;  // set when a CTA gave up waiting for a tile

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
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

// Shared-memory tile at `src` to the 4-D box of `map` at (c0, c1, c2, c3) (all >= 0; parts
// outside the tensor are not written), as one bulk group of the calling thread.
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2, int c3) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];\n" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

// Named barrier 2 over the 128 epilogue threads of the tcgen05 kernel; the _all form also
// returns whether `v` holds in every one of them.
__device__ __forceinline__ void epilogue_sync() { asm volatile("bar.sync 2, 128;\n" ::: "memory"); }
__device__ __forceinline__ bool epilogue_all(bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 2, 128, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)v)
      : "memory");
  return r != 0;
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

__device__ __forceinline__ void ldsm_x4_trans(unsigned* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

// Address of the 16-byte chunk `chunk` of halo pixel p in a tile written by TMA with the
// 64-byte swizzle.
__device__ __forceinline__ const unsigned char* swz(const unsigned char* tile, int p, int chunk) {
  return tile + p * 64 + ((chunk ^ ((p >> 1) & 3)) << 4);
}

// Persistent loop over the 8 x 16 tiles of a [B][H][W] grid; tile i of this CTA uses slot
// i & 1.  One tile ahead of its use, thread 0 arms bar[slot] with `bytes` and issue(b, y0,
// x0, slot) starts the tile's TMA copies (none when bytes == 0), and every thread runs
// prefetch(b, y0, x0), plain loads into registers.  commit() moves those registers into
// shared memory once the previous tile is done with it, and body(b, y0, x0, slot) runs when
// the copies have landed.  Returns false, with the timeout flag set, if a wait gave up (after
// a bounded wait for the copy still in flight).  bar[] must be initialised, and the
// initialisation made visible by a barrier, before the call.
template <class Issue, class Prefetch, class Commit, class Body>
__device__ __forceinline__ bool tile_loop(int B, int H, int W, uint64_t* bar, unsigned bytes, Issue issue,
                                          Prefetch prefetch, Commit commit, Body body) {
  // 32-bit tile arithmetic: the host rejects grids of 2^31 pixels or more
  const unsigned tilesx = (W + TX - 1) / TX, tpi = tilesx * ((H + TY - 1) / TY);
  const unsigned ntiles = (unsigned)B * tpi;
  auto coords = [&](unsigned tile, int& b, int& y0, int& x0) {
    const unsigned bb = tile / tpi, rr = tile - bb * tpi, ty = rr / tilesx;
    b = (int)bb;
    y0 = (int)ty * TY;
    x0 = (int)(rr - ty * tilesx) * TX;
  };
  auto start = [&](unsigned tile, int s) {
    int b, y0, x0;
    coords(tile, b, y0, x0);
    if (bytes != 0 && threadIdx.x == 0) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic reads of the slot come first
      mbar_expect_tx(&bar[s], bytes);
      issue(b, y0, x0, s);
    }
    prefetch(b, y0, x0);
  };
  if (blockIdx.x < ntiles) {
    start(blockIdx.x, 0);
    commit();
  }
  int i = 0;
  for (unsigned tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
    const int s = i & 1;
    const unsigned next = tile + gridDim.x;
    if (next < ntiles) start(next, s ^ 1);  // slot s^1 was released by the barrier ending the previous tile
    const bool ok = bytes == 0 || mbar_wait(&bar[s], (unsigned)((i >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(&g_lpd_timeout, 1);
      if (bytes != 0 && next < ntiles) mbar_wait(&bar[s ^ 1], (unsigned)(((i + 1) >> 1) & 1));
      return false;
    }
    int b, y0, x0;
    coords(tile, b, y0, x0);
    body(b, y0, x0, s);
    __syncthreads();
    if (next < ntiles) commit();
  }
  return true;
}

// One thread waits, bounded by `tries`, on an mbarrier that nothing arrives on: the wait
// gives up, records the timeout in the flag tat_lpd_check reads, and returns.  It exercises
// the give-up path of the convolutions' waits without a stuck copy.
__global__ void k_wait_probe(int tries, int* gave_up) {
  __shared__ uint64_t bar;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  bool ok = false;
  for (int i = 0; i < tries && !ok; ++i) ok = mbar_try_wait(&bar, 0u);
  if (!ok) atomicExch(&g_lpd_timeout, 1);
  *gave_up = ok ? 0 : 1;
}

__device__ __forceinline__ void init_bars(uint64_t* bar) {
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
}

// One 8 x 16 output tile of the mid layer from a staged halo (and, with MASK, the
// staged ReLU mask) and the staged weights.
// FWD: out = relu(conv(in) + b).  BWD (data gradient): out = conv^T(g * [h > 0]),
// i.e. the same implicit GEMM with the taps flipped and in/out channels swapped;
// without MASK the gradient arrives already masked.  With OMASK the output is
// multiplied by [h_in > 0] from the staged halo `otile` (the gradient of the
// previous layer's pre-activation).
template <bool BWD, bool MASK, bool OMASK>
__device__ __forceinline__ void mid_tile(const unsigned char* tile, const unsigned char* mtile,
                                         const unsigned char* otile, const tat_bf16* wsm,
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
      if (MASK) {
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
    const int p = (warp + 1) * XW + g + 8 * half + 1;  // this pixel in a staged halo
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int co = nt * 8 + 2 * t;
      float v0 = acc[nt][2 * half], v1 = acc[nt][2 * half + 1];
      if (!BWD) {
        v0 = fmaxf(v0 + bias[co], 0.f);
        v1 = fmaxf(v1 + bias[co + 1], 0.f);
      }
      unsigned v = (unsigned)tobf(v0) | ((unsigned)tobf(v1) << 16);
      if (OMASK) v = relu_masked(v, *reinterpret_cast<const unsigned*>(swz(otile, p, nt) + 4 * t));
      *reinterpret_cast<unsigned*>(dst + co) = v;
    }
  }
}

// Dynamic shared memory of the mid-layer kernel: alignment slack, two stages of NT
// tiles (value tile, the mask tile with MASK, the output-mask tile with OMASK), the
// padded weights, two mbarriers.
template <int NT>
constexpr size_t mid_smem_bytes() {
  return 1024 + 2 * NT * HALO_SLOT + 9 * C * CP * 2 + 2 * sizeof(uint64_t);
}

// BF16 element k (0..7) of a 16-byte word.
__device__ __forceinline__ tat_bf16 bf16_of(const uint4& v, int k) {
  const unsigned word = k < 2 ? v.x : k < 4 ? v.y : k < 6 ? v.z : v.w;
  return (tat_bf16)((k & 1) ? word >> 16 : word & 0xffffu);
}

// Stages the 32 -> 32 weights w[tap][co][ci] (16-byte aligned) in shared memory with 16-byte
// loads, all of a thread's loads in flight before its first store.  Word u of w holds the
// input channels ci = 8 (u mod 4) .. + 7 of (tap, co) = (u / 128, (u / 4) mod 32); `place`
// stores it.  Threads t = 0 .. NTHR - 1 of the calling group take part.
template <int NTHR, class Place>
__device__ __forceinline__ void stage_mid_weights(const tat_bf16* __restrict__ w, int t, Place place) {
  constexpr int NV = 9 * C * C / 8, PER = (NV + NTHR - 1) / NTHR;
  const uint4* w4 = reinterpret_cast<const uint4*>(w);
  uint4 v[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int u = t + NTHR * i;
    if (u < NV) v[i] = __ldg(w4 + u);
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int u = t + NTHR * i;
    if (u < NV) place(u >> 7, (u >> 2) & 31, u & 3, v[i]);
  }
}

template <bool BWD, bool MASK, bool OMASK>
__global__ void __launch_bounds__(256) k_conv_mid(int B, int H, int W, const __grid_constant__ CUtensorMap map_in,
                                                  const __grid_constant__ CUtensorMap map_mask,
                                                  const __grid_constant__ CUtensorMap map_omask,
                                                  const tat_bf16* __restrict__ w, const float* __restrict__ bias,
                                                  tat_bf16* __restrict__ out) {
  TAT_GRID_DEPENDENCY();
  extern __shared__ unsigned char dsm[];
  unsigned char* sm = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);  // 1024-aligned (swizzle period)
  constexpr int NT = 1 + MASK + OMASK;
  constexpr int OT = (1 + MASK) * HALO_SLOT;  // offset of the output-mask tile in a stage
  constexpr int STAGE = NT * HALO_SLOT;
  tat_bf16* wsm = reinterpret_cast<tat_bf16*>(sm + 2 * STAGE);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * STAGE + 9 * C * CP * 2);
  // weights: wsm[tap][n][k] with n the output channel of this GEMM and k its input channel
  stage_mid_weights<256>(w, threadIdx.x, [&](int tap, int co, int j, const uint4& v) {
    if (BWD) {
#pragma unroll
      for (int k = 0; k < 8; ++k) wsm[((8 - tap) * C + 8 * j + k) * CP + co] = bf16_of(v, k);
    } else {
      reinterpret_cast<uint4*>(wsm)[(tap * C + co) * (CP / 8) + j] = v;
    }
  });
  init_bars(bar);
  __syncthreads();
  tile_loop(
      B, H, W, bar, NT * HALO_BYTES,
      [&](int b, int y0, int x0, int s) {
        tma_load_4d(sm + s * STAGE, &map_in, 0, x0 - 1, y0 - 1, b, &bar[s]);
        if (MASK) tma_load_4d(sm + s * STAGE + HALO_SLOT, &map_mask, 0, x0 - 1, y0 - 1, b, &bar[s]);
        if (OMASK) tma_load_4d(sm + s * STAGE + OT, &map_omask, 0, x0 - 1, y0 - 1, b, &bar[s]);
      },
      [](int, int, int) {}, [] {},
      [&](int b, int y0, int x0, int s) {
        mid_tile<BWD, MASK, OMASK>(sm + s * STAGE, sm + s * STAGE + HALO_SLOT, sm + s * STAGE + OT, wsm, bias, out, b,
                                   y0, x0, H, W);
      });
}

// ---- 32 -> 32 forward on the 5th-generation tensor cores (tcgen05, accumulators in TMEM)
//
// Implicit GEMM per tile of 16 rows x 8 pixels: M = 128 pixels, N = 32 output channels,
// K = 9 taps x 32 input channels in 18 tcgen05.mma (kind::f16, BF16 operands, FP32
// accumulation) issued by one thread.  The halo of a tile (18 x 10 pixels of 32 channels)
// arrives by one TMA copy with the 64-byte swizzle: [pixel][64 B], the 16-byte chunks of a
// pixel permuted by address bits 7-8.  It is the A operand as it lies, in the canonical
// K-major layout with the same swizzle: a row (pixel) is 64 B = the whole K of one tap, the
// tap's A is the halo shifted by the tap's offset (start address + 64 B per pixel; the
// swizzle follows the absolute address, so odd shifts read what the copy wrote), 8-row
// groups 640 B apart (one halo row of 10 pixels), the second K = 16 step 32 B further.  The
// weights (B) use the layout without swizzle: 8 x 16-byte core matrices of 8 output channels
// x 8 input channels.  The accumulator of a
// tile is 32 TMEM columns; two of them alternate, so the epilogue of tile i-1 (tcgen05.ld,
// bias, ReLU, BF16 into a shared-memory tile that one bulk tensor store writes out) overlaps
// the MMAs of tile i, and two halo slots alternate, so the halo of tile i+1 loads meanwhile.
// The weights are staged by the MMA and epilogue warps while the first halos load.
// tcgen05.commit signals on an
// mbarrier when a tile's MMAs have finished reading their halo slot and writing their
// accumulator.  Every wait is bounded; on a timeout the CTA records it, waits (bounded) for
// its copies and MMAs in flight, frees its TMEM and returns.
namespace tc {
constexpr int TX = 8, TY = 16;             // tile: M = 128 pixels
constexpr int HX = TX + 2, HY = TY + 2;    // 10 x 18 halo
constexpr int SLOT = 11776;                // one staged halo [180 pixels][64 B], a multiple of the 512-byte
                                           // swizzle period
constexpr int NS = 2;                      // halo slots: tile n+1 loads while tile n computes
constexpr int HALO_TX = HX * HY * 64;      // bytes of a halo
constexpr int WOFF = NS * SLOT;            // weights [tap][plane][co][16 B], 2 KB per tap
constexpr int BOFF = WOFF + 9 * 2048;      // bias, 32 floats
constexpr int OOFF = BOFF + 128;           // output tile [16][8][32] BF16 for the bulk store, 8 KB
constexpr int NACC = 2;                    // accumulators in TMEM: the MMAs run up to NACC - 1 tiles ahead
constexpr int CTAS = 4;                    // resident CTAs per SM (shared memory, TMEM: CTAS x TMEM_COLS <= 512)
constexpr int MOFF = OOFF + TX * TY * 64;  // mbarriers: halo full[NS], empty[NS], accumulator full[NACC],
                                           // empty[NACC]; then the TMEM address
constexpr int SMEM = 512 + MOFF + 256;     // alignment slack (512 B: the swizzled halos) + the layout above
                                           // (49.5 KB: 4 CTAs per SM)
constexpr int TMEM_COLS = 32 * NACC;       // NACC accumulators of 32 FP32 columns (a power of 2 >= 32)
static_assert(2 * (NS + NACC) * 8 + 4 <= 256, "mbarrier region");
static_assert(CTAS * TMEM_COLS <= 512, "TMEM columns of the resident CTAs");
// Instruction descriptor (kind::f16): FP32 D, BF16 A and B, both K-major, N = 32, M = 128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
}  // namespace tc

// Shared-memory matrix descriptor: canonical K-major layout without swizzle, start address,
// leading byte offset (between the two core matrices along K) and stride byte offset
// (between core-matrix groups along M or N), all in 16-byte units; version 1.  OR-ing
// kSwizzle64 into it selects the 64-byte-swizzle layout (rows of 64 B, SBO between 8-row
// groups, LBO unused).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}
constexpr uint64_t kSwizzle64 = 4ull << 61;  // layout type field: 64-byte swizzle

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 32 consecutive FP32 columns of the warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// FWD: out = relu(conv(in) + b).  BWD: out = conv^T(in) (the data gradient of an already
// masked gradient `in`: taps flipped, input and output channels swapped), times [omask > 0]
// with OMASK (the ReLU mask of the layer below).
//
// Warp roles (192 threads): warp 0 loads halos (TMA), warp 1 owns the TMEM and issues the
// MMAs, warps 2-5 run the epilogue (warp w reads TMEM lanes 32 (w mod 4) .. + 31).  They hand
// tiles over through mbarriers only -- halo full / empty per slot, accumulator full / empty
// per TMEM buffer -- so no CTA-wide barrier sits inside the tile loop.
template <bool BWD, bool OMASK>
__global__ void __launch_bounds__(192, tc::CTAS) k_conv_mid_tc(int B, int H, int W, const __grid_constant__ CUtensorMap map8,
                                                        const __grid_constant__ CUtensorMap map_out,
                                                        const tat_bf16* __restrict__ w, const float* __restrict__ bias,
                                                        const tat_bf16* __restrict__ omask) {
  TAT_GRID_DEPENDENCY();
  constexpr int TX = tc::TX, TY = tc::TY, HX = tc::HX, SLOT = tc::SLOT, WOFF = tc::WOFF;
  constexpr int BOFF = tc::BOFF, MOFF = tc::MOFF, HALO_TX = tc::HALO_TX, TMEM_COLS = tc::TMEM_COLS, NS = tc::NS;
  constexpr int NACC = tc::NACC;
  constexpr uint32_t IDESC = tc::IDESC;
  extern __shared__ unsigned char dsm[];
  unsigned char* sm = dsm + ((512u - (smem_u32(dsm) & 511u)) & 511u);
  tat_bf16* wsm = reinterpret_cast<tat_bf16*>(sm + WOFF);
  float* bsm = reinterpret_cast<float*>(sm + BOFF);
  uint4* osm = reinterpret_cast<uint4*>(sm + tc::OOFF);     // [pixel][4 x 16 B]
  uint64_t* hfull = reinterpret_cast<uint64_t*>(sm + MOFF);  // [NS] halo landed
  uint64_t* hempty = hfull + NS;                              // [NS] halo consumed by the MMAs
  uint64_t* afull = hempty + NS;                              // [NACC] accumulator written
  uint64_t* aempty = afull + NACC;                            // [NACC] accumulator read by the epilogue
  uint32_t* tslot = reinterpret_cast<uint32_t*>(aempty + NACC);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int k = 0; k < NS; ++k) {
      mbar_init(&hfull[k], 1);
      mbar_init(&hempty[k], 1);
    }
    for (int k = 0; k < NACC; ++k) {
      mbar_init(&afull[k], 1);
      mbar_init(&aempty[k], 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  if (warp != 0) {
    // Warps 1-5 stage the weights w[tap][co][ci] -> B[tap][k / 8][n][k % 8] (n the output
    // channel of this GEMM, k its input channel; BWD: n = ci, k = co, tap mirrored) and the
    // bias while warp 0 already loads the first halos; a named barrier among the 160 threads
    // orders the stores (made visible to the MMAs' async proxy) before the first MMA.
    stage_mid_weights<160>(w, tid - 32, [&](int tap, int co, int j, const uint4& v) {
      if (BWD) {
#pragma unroll
        for (int k = 0; k < 8; ++k) wsm[(8 - tap) * 1024 + (co >> 3) * 256 + (8 * j + k) * 8 + (co & 7)] = bf16_of(v, k);
      } else {
        reinterpret_cast<uint4*>(wsm)[tap * 128 + j * 32 + co] = v;
      }
    });
    if (!BWD && tid - 32 < C) bsm[tid - 32] = bias[tid - 32];
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("bar.sync 1, 160;\n" ::: "memory");
  }
  const uint32_t sbase = smem_u32(sm);
  // 32-bit tile arithmetic: the host rejects grids of 2^31 pixels or more
  const unsigned tilesx = (W + TX - 1) / TX, tpi = tilesx * ((H + TY - 1) / TY);
  const unsigned ntiles = (unsigned)B * tpi;
  const int mine = ntiles > blockIdx.x ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;  // tiles of this CTA
  auto coords = [&](int n, int& b, int& y0, int& x0) {
    const unsigned tile = blockIdx.x + (unsigned)n * gridDim.x, bb = tile / tpi, rr = tile - bb * tpi,
                   ty = rr / tilesx;
    b = (int)bb;
    y0 = (int)ty * TY;
    x0 = (int)(rr - ty * tilesx) * TX;
  };
  bool ok = true;
  if (warp == 0) {
    if (lane == 0) {  // halo loads
      int issued = 0;
      for (int n = 0; n < mine && ok; ++n) {
        const int k = n % NS;
        if (n >= NS) ok = mbar_wait(&hempty[k], (unsigned)((n / NS + 1) & 1));  // MMAs of tile n - NS done
        if (!ok) break;
        int b, y0, x0;
        coords(n, b, y0, x0);
        mbar_expect_tx(&hfull[k], HALO_TX);
        tma_load_4d(sm + k * SLOT, &map8, 0, x0 - 1, y0 - 1, b, &hfull[k]);
        issued = n + 1;
      }
      if (!ok) {  // let the copies in flight land (their slots are not reused after this)
        for (int n = issued - NS > 0 ? issued - NS : 0; n < issued; ++n)
          mbar_wait(&hfull[n % NS], (unsigned)((n / NS) & 1));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMAs
      int committed = 0;
      for (int n = 0; n < mine && ok; ++n) {
        const int k = n % NS, a = n % NACC;
        ok = mbar_wait(&hfull[k], (unsigned)((n / NS) & 1));
        if (ok && n >= NACC) ok = mbar_wait(&aempty[a], (unsigned)((n / NACC + 1) & 1));  // tile n-NACC read out
        if (!ok) break;
        tc_fence_after();
        const uint32_t d = tbase + (uint32_t)(a * 32);
        const uint32_t abase = sbase + k * SLOT, wbase = sbase + WOFF;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const int dy = tap / 3, dx = tap % 3;
#pragma unroll
          for (int kc = 0; kc < 2; ++kc) {
            const uint64_t ad = umma_desc(abase + (dy * HX + dx) * 64 + 32 * kc, 16, HX * 64) | kSwizzle64;
            const uint64_t bd = umma_desc(wbase + tap * 2048 + 2 * kc * 512, 512, 128);
            umma_f16(d, ad, bd, IDESC, (tap | kc) != 0);
          }
        }
        umma_commit(&hempty[k]);  // halo slot free once these MMAs have read it
        umma_commit(&afull[a]);   // accumulator ready
        committed = n + 1;
      }
      if (!ok && committed > 0)  // the MMAs in flight must finish before the TMEM is freed
        mbar_wait(&afull[(committed - 1) % NACC], (unsigned)(((committed - 1) / NACC) & 1));
    }
  } else {  // epilogue: 128 threads, thread m of the tile = TMEM lane m = pixel (m / 8, m % 8)
    const int quarter = warp & 3;
    const int m = 32 * quarter + lane;
    for (int n = 0; n < mine; ++n) {
      const int a = n % NACC;
      int b, y0, x0;
      coords(n, b, y0, x0);
      // OMASK: the mask of the tile's 16-byte chunks m, m + 128, m + 256, m + 384 (pixel
      // chunk / 4, part chunk mod 4: a warp reads 512 contiguous bytes per load), issued before
      // the wait for the accumulator so that their latency overlaps it
      uint4 mk[4];
      if (OMASK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int ch = m + 128 * i, pm = ch >> 2;
          const int y = y0 + (pm >> 3), x = x0 + (pm & 7);
          mk[i] = y < H && x < W
                      ? reinterpret_cast<const uint4*>(omask + (((long long)b * H + y) * W + x) * C)[ch & 3]
                      : make_uint4(0u, 0u, 0u, 0u);
        }
      }
      ok = mbar_wait(&afull[a], (unsigned)((n / NACC) & 1));
      ok = epilogue_all(ok);  // one decision for the four warps, which meet at named barriers below
      if (!ok) break;
      tc_fence_after();
      uint32_t r[32];
      tmem_ld32(tbase + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(a * 32), r);
      tc_fence_before();
      mbar_arrive(&aempty[a]);
      uint4 pk[4];  // channels 8q .. 8q+7 of this pixel, BF16
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        unsigned wd[4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const int c0 = 8 * q + 2 * kk;
          float v0 = __uint_as_float(r[c0]), v1 = __uint_as_float(r[c0 + 1]);
          if (!BWD) {
            v0 = fmaxf(v0 + bsm[c0], 0.f);
            v1 = fmaxf(v1 + bsm[c0 + 1], 0.f);
          }
          wd[kk] = (unsigned)tobf(v0) | ((unsigned)tobf(v1) << 16);
        }
        pk[q] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
      }
      // the previous tile's bulk store has finished reading the staging tile
      if (m == 0) asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
      epilogue_sync();
      // chunk (q + m / 2) mod 4 in step q: the 8 lanes of a 128-byte wavefront write 8
      // different bank groups
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = (q + (m >> 1)) & 3;
        osm[4 * m + c] = c == 0 ? pk[0] : c == 1 ? pk[1] : c == 2 ? pk[2] : pk[3];
      }
      if (OMASK) {  // mask the staged tile chunk by chunk, as the mask was read
        epilogue_sync();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          uint4& o = osm[m + 128 * i];
          o = make_uint4(relu_masked(o.x, mk[i].x), relu_masked(o.y, mk[i].y), relu_masked(o.z, mk[i].z),
                         relu_masked(o.w, mk[i].w));
        }
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // generic writes, read by the bulk store
      epilogue_sync();
      if (m == 0) tma_store_4d(&map_out, osm, 0, x0, y0, b);  // pixels outside the image are clipped
    }
    if (m == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
  }
  if (!ok) atomicExch(&g_lpd_timeout, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
}

// ---- 32 -> 32 weight gradient on tcgen05 (an already masked gradient G')
//
// dW[tap][co][ci] = sum_p G'(p)[co] in(p + tap)[ci] is a GEMM with K = pixels, whose
// M = 32 output channels are below the 64 / 128 rows of an MMA; so the M rows stack four
// copies of G' shifted by j = 0..3 pixels along x (both operands MN-major: a pixel's 32
// channels are one 64-byte row of the swizzled halo, and the four M atoms are 64 B = one
// pixel apart).  With B = in shifted by (dy - 1, +1), rows (j, co) of chain dy sum
// G'(Q)[co] in(Q + (dy - 1, 1 - j))[ci] over Q = P + (0, j), P the tile's pixels: the taps
// (dy, dx = 2 - j) for j = 0, 1, 2 (j = 3 is not used).  The three dy share A: they are the
// three N atoms of one MMA (N = 96, atoms one in-box row apart).  So that Q still covers
// every pixel of the image once, the tile columns start one tile left of the image (x0 = -8;
// the copies fill zeros outside it).  Per 16 x 8-pixel tile: 8 MMAs of M = 128, N = 96,
// K = 16, accumulated in TMEM over all tiles of the CTA; warp 0 streams the two halos (G'
// 16 x 11 pixels, in 18 x 8) by TMA, warp 1 issues the MMAs, warps 2-5 add up db from the G'
// halo meanwhile (a stage is free once both are done with it) and read the sums out once at
// the end into the per-CTA partials [tap][co][ci] then [co].  Every wait is bounded.
namespace wg {
constexpr int TX = 8, TY = 16;
constexpr int GX = TX + 3, GY = TY;                   // G' box: pixels x0 .. x0+10, rows y0 .. y0+15
constexpr int IX = TX, IY = TY + 2;                   // in box: pixels x0+1 .. x0+8, rows y0-1 .. y0+16
constexpr int GSZ = 11264, ISZ = 9216;                // 176 and 144 pixels of 64 B (multiples of 512 B)
constexpr int SLOT = GSZ + ISZ;                       // one stage
constexpr int NS = 4;                                 // stages
constexpr int MOFF = NS * SLOT;                       // mbarriers full[NS], empty[NS], done; TMEM address
constexpr int SMEM = 512 + MOFF + 128;
constexpr int TMEM_COLS = 128;                        // D: columns 32 dy + ci (96 used)
constexpr int CTAS = 152;                             // one per SM: fewer partial sets to add up
// kind::f16, FP32 D, BF16 A and B, both MN-major (bits 15, 16), N = 96, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((96u >> 3) << 17) |
                           ((128u >> 4) << 24);
}  // namespace wg

__global__ void __launch_bounds__(192, 1) k_conv_mid_wgrad_tc(int B, int H, int W,
                                                              const __grid_constant__ CUtensorMap map_g,
                                                              const __grid_constant__ CUtensorMap map_in,
                                                              float* __restrict__ partial) {
  TAT_GRID_DEPENDENCY();
  constexpr int NS = wg::NS, SLOT = wg::SLOT, GSZ = wg::GSZ, TMEM_COLS = wg::TMEM_COLS;
  extern __shared__ unsigned char dsm[];
  unsigned char* sm = dsm + ((512u - (smem_u32(dsm) & 511u)) & 511u);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + wg::MOFF);
  uint64_t* empty = full + NS;
  uint64_t* done = empty + NS;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ float dbred[4][C];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int k = 0; k < NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1 + 128);  // the MMAs' commit and the 128 db threads
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t sbase = smem_u32(sm);
  // tiles: image b, tile row ty, tile column tx with x0 = 8 (tx - 1), tx = 0 .. ceil(W / 8)
  const unsigned tilesx = (W + wg::TX - 1) / wg::TX + 1, tpi = tilesx * ((H + wg::TY - 1) / wg::TY);
  const unsigned ntiles = (unsigned)B * tpi;
  const int mine = ntiles > blockIdx.x ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;
  auto coords = [&](int n, int& b, int& y0, int& x0) {
    const unsigned tile = blockIdx.x + (unsigned)n * gridDim.x, bb = tile / tpi, rr = tile - bb * tpi,
                   ty = rr / tilesx;
    b = (int)bb;
    y0 = (int)ty * wg::TY;
    x0 = ((int)(rr - ty * tilesx) - 1) * wg::TX;
  };
  bool ok = true;
  if (warp == 0) {
    if (lane == 0) {  // halo loads
      int issued = 0;
      for (int n = 0; n < mine && ok; ++n) {
        const int k = n % NS;
        if (n >= NS) ok = mbar_wait(&empty[k], (unsigned)((n / NS + 1) & 1));  // MMAs of tile n - NS done
        if (!ok) break;
        int b, y0, x0;
        coords(n, b, y0, x0);
        mbar_expect_tx(&full[k], (wg::GX * wg::GY + wg::IX * wg::IY) * 64);
        tma_load_4d(sm + k * SLOT, &map_g, 0, x0, y0, b, &full[k]);
        tma_load_4d(sm + k * SLOT + GSZ, &map_in, 0, x0 + 1, y0 - 1, b, &full[k]);
        issued = n + 1;
      }
      if (!ok)  // let the copies in flight land (their slots are not reused after this)
        for (int n = issued - NS > 0 ? issued - NS : 0; n < issued; ++n)
          mbar_wait(&full[n % NS], (unsigned)((n / NS) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMAs
      for (int n = 0; n < mine && ok; ++n) {
        const int k = n % NS;
        ok = mbar_wait(&full[k], (unsigned)((n / NS) & 1));
        if (!ok) break;
        tc_fence_after();
        const uint32_t gb = sbase + k * SLOT, ib = gb + GSZ;
#pragma unroll
        for (int st = 0; st < wg::TY / 2; ++st) {  // K = 16 pixels = tile rows 2 st, 2 st + 1
          // A: G' from pixel (2 st, 0) of the G' box; M atoms one pixel apart, 8-row groups one box row apart.
          // B: in from row 2 st of the in box (rows y0 - 1 ..); N atoms (dy) and 8-row groups one box row apart.
          const uint64_t ad = umma_desc(gb + 2 * st * wg::GX * 64, 64, wg::GX * 64) | kSwizzle64;
          const uint64_t bd = umma_desc(ib + 2 * st * wg::IX * 64, wg::IX * 64, wg::IX * 64) | kSwizzle64;
          umma_f16(tbase, ad, bd, wg::IDESC, (n | st) != 0);
        }
        umma_commit(&empty[k]);  // stage free once these MMAs have read it
      }
    }
    if (lane == 0) {
      umma_commit(done);        // arrives once every MMA issued so far has completed
      mbar_wait(done, 0u);      // (bounded) none is in flight when the TMEM is freed
    }
  } else {
    // db: thread t = co + 32 r adds G'(ky, kx)[co] over the tile rows ky = 4 r .. 4 r + 3 of every
    // tile (its own 8 columns; zeros outside the image)
    const int t = tid - 64, co = t & 31, r4 = t >> 5;
    float db = 0.f;
    for (int n = 0; n < mine && ok; ++n) {
      const int k = n % NS;
      ok = mbar_wait(&full[k], (unsigned)((n / NS) & 1));
      if (!ok) break;
      const unsigned char* gt = sm + k * SLOT;
#pragma unroll
      for (int ky = 4 * r4; ky < 4 * r4 + 4; ++ky)
#pragma unroll
        for (int kx = 0; kx < 8; ++kx) {
          const int p = ky * wg::GX + kx;
          db += bf(*reinterpret_cast<const tat_bf16*>(swz(gt, p, co >> 3) + 2 * (co & 7)));
        }
      mbar_arrive(&empty[k]);
    }
    dbred[r4][co] = db;
    // read-out: warp w reads TMEM lanes 32 (w mod 4) .. + 31 = rows (j = w mod 4, co = lane)
    const int j = warp & 3;
    const bool fin = mbar_wait(done, 0u);
    ok = __all_sync(0xffffffffu, fin && ok);
    tc_fence_after();
    float* out = partial + (size_t)blockIdx.x * (9 * C * C + C);
    if (j < 3) {
#pragma unroll 1
      for (int dy = 0; dy < 3; ++dy) {
        uint32_t r[32];
        tmem_ld32(tbase + ((uint32_t)(32 * j) << 16) + (uint32_t)(32 * dy), r);
        float* dst = out + ((3 * dy + 2 - j) * C + lane) * C;  // dW[tap = 3 dy + dx][co][ci], dx = 2 - j
#pragma unroll
        for (int ci = 0; ci < C; ++ci) dst[ci] = mine > 0 ? __uint_as_float(r[ci]) : 0.f;
      }
    }
    asm volatile("bar.sync 2, 128;\n" ::: "memory");  // dbred complete
    if (t < C) out[9 * C * C + t] = dbred[0][t] + dbred[1][t] + dbred[2][t] + dbred[3][t];
  }
  if (!ok) atomicExch(&g_lpd_timeout, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(TMEM_COLS) : "memory");
}

// Dynamic shared memory of k_conv_mid_wgrad: alignment slack, two slots of three halos
// (input, gradient, forward output -- the last unused when the gradient arrives masked),
// two mbarriers.
constexpr size_t wgrad_smem_bytes() { return 1024 + 2 * 3 * HALO_SLOT + 2 * sizeof(uint64_t); }

// dW[tap][co][ci] = sum_p G'(p)[co] in(p + tap)[ci], db[co] = sum_p G'(p)[co],
// G' = g * [h_out > 0] (or g itself, already masked, without MASK).  9 warps, warp w =
// tap w: per tile row a K = 16 step with A = G'^T (ldmatrix.trans of the g and h_out
// halos, masked in registers) and
// B = the input row shifted by the tap; warp 0 also multiplies A by a column of
// ones for db.  The three halos of the next tile arrive by TMA meanwhile.
// Per-CTA partials [tap][co][ci] then [co].
template <bool MASK>
__global__ void __launch_bounds__(288, 2) k_conv_mid_wgrad(int B, int H, int W, const __grid_constant__ CUtensorMap map_in,
                                                           const __grid_constant__ CUtensorMap map_g,
                                                           const __grid_constant__ CUtensorMap map_h,
                                                           float* __restrict__ partial) {
  TAT_GRID_DEPENDENCY();
  constexpr int STAGE = 3 * HALO_SLOT;
  extern __shared__ unsigned char dsm[];
  unsigned char* sm = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * STAGE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int dy = warp / 3, dx = warp % 3, m = lane >> 3;
  init_bars(bar);
  __syncthreads();
  float acc[2][4][4], accb[2][4];
#pragma unroll
  for (int mh = 0; mh < 2; ++mh) {
#pragma unroll
    for (int k = 0; k < 4; ++k) accb[mh][k] = 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[mh][nt][k] = 0.f;
  }
  const unsigned ones[2] = {0x3f803f80u, 0x3f803f80u};
  const bool ok = tile_loop(
      B, H, W, bar, (MASK ? 3 : 2) * HALO_BYTES,
      [&](int b, int y0, int x0, int s) {
        unsigned char* slot = sm + s * STAGE;
        tma_load_4d(slot, &map_in, 0, x0 - 1, y0 - 1, b, &bar[s]);
        tma_load_4d(slot + HALO_SLOT, &map_g, 0, x0 - 1, y0 - 1, b, &bar[s]);
        if (MASK) tma_load_4d(slot + 2 * HALO_SLOT, &map_h, 0, x0 - 1, y0 - 1, b, &bar[s]);
      },
      [](int, int, int) {}, [] {},
      [&](int, int, int, int s) {
        const unsigned char* it = sm + s * STAGE;
        const unsigned char* gt = it + HALO_SLOT;
        const unsigned char* ht = it + 2 * HALO_SLOT;
#pragma unroll 2
        for (int row = 0; row < TY; ++row) {
          unsigned a[2][4];
#pragma unroll
          for (int mh = 0; mh < 2; ++mh) {
            // matrices (co 0-7, px 0-7), (co 8-15, px 0-7), (co 0-7, px 8-15), (co 8-15, px 8-15) of G'^T
            const int p = (row + 1) * XW + 1 + (m >> 1) * 8 + (lane & 7);
            ldsm_x4_trans(a[mh], swz(gt, p, 2 * mh + (m & 1)));
            if (MASK) {
              unsigned mk[4];
              ldsm_x4_trans(mk, swz(ht, p, 2 * mh + (m & 1)));
#pragma unroll
              for (int j = 0; j < 4; ++j) a[mh][j] = relu_masked(a[mh][j], mk[j]);
            }
          }
#pragma unroll
          for (int np = 0; np < 2; ++np) {
            // matrices (ci of n-tile 2np, px 0-7), (2np, px 8-15), (2np+1, px 0-7), (2np+1, px 8-15)
            const int p = (row + dy) * XW + dx + (m & 1) * 8 + (lane & 7);
            unsigned bq[4];
            ldsm_x4_trans(bq, swz(it, p, 2 * np + (m >> 1)));
#pragma unroll
            for (int mh = 0; mh < 2; ++mh) {
              mma_bf16(acc[mh][2 * np], a[mh], bq);
              mma_bf16(acc[mh][2 * np + 1], a[mh], bq + 2);
            }
          }
          if (warp == 0) {
            mma_bf16(accb[0], a[0], ones);
            mma_bf16(accb[1], a[1], ones);
          }
        }
      });
  if (!ok) return;
  constexpr int NW = 9 * C * C + C;
  float* pp = partial + (size_t)blockIdx.x * NW;
#pragma unroll
  for (int mh = 0; mh < 2; ++mh)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int co = mh * 16 + g, ci = nt * 8 + 2 * t;
      float* d0 = pp + (warp * C + co) * C + ci;
      float* d1 = pp + (warp * C + co + 8) * C + ci;
      d0[0] = acc[mh][nt][0];
      d0[1] = acc[mh][nt][1];
      d1[0] = acc[mh][nt][2];
      d1[1] = acc[mh][nt][3];
    }
  if (warp == 0 && t == 0) {
#pragma unroll
    for (int mh = 0; mh < 2; ++mh) {
      pp[9 * C * C + mh * 16 + g] = accb[mh][0];
      pp[9 * C * C + mh * 16 + g + 8] = accb[mh][2];
    }
  }
}

// ------------------------------------------------------------------ thin layers (tensor cores)
//
// The in layer (cin = 2 or 3 planes -> 32) and the out layer (32 -> 1) are implicit GEMMs too,
// with one dimension of 8 to 27: mma.sync m16n8k16 on 8 x 16 pixel tiles, one warp per tile
// row, persistent CTAs.  BF16 x BF16 products are exact in FP32, so the tensor cores give the
// sums the CUDA cores would, in another order.  An FP32 operand (the gradient of the out
// layer's output) enters as two BF16 terms hi + lo, hi = bf16(v), lo = bf16(v - hi), which
// carry 16 of its 24 significand bits (relative error below 2^-16 per product).

// Halo of CIN FP32 planes around a tile, prefetched into registers (kXPer values per thread)
// and committed to shared memory as BF16.
constexpr int kXPer = (3 * XH * XW + 255) / 256;

__device__ __forceinline__ const float* pick(int c, const float* p0, const float* p1, const float* p2) {
  return c == 0 ? p0 : (c == 1 ? p1 : p2);
}

template <int CIN>
__device__ __forceinline__ void x_prefetch(float* v, const float* x0, const float* x1, const float* x2, int b,
                                           int y0, int x0c, int H, int W) {
#pragma unroll
  for (int k = 0; k < kXPer; ++k) {
    const int e = threadIdx.x + 256 * k;
    v[k] = 0.f;
    if (e < CIN * XH * XW) {
      const int c = e / (XH * XW), r = (e / XW) % XH, j = e % XW;
      const int yy = y0 - 1 + r, xx = x0c - 1 + j;
      if (yy >= 0 && yy < H && xx >= 0 && xx < W) v[k] = pick(c, x0, x1, x2)[((long long)b * H + yy) * W + xx];
    }
  }
}

// h = relu(conv_in(x) + b): A[pixel][k = tap * CIN + c] gathered from the BF16 halo (K padded
// to 32), B = w[k][co] held in registers, N = 32.
template <int CIN>
__global__ void __launch_bounds__(256) k_conv_in_fwd(int B, int H, int W, const float* __restrict__ x0,
                                                     const float* __restrict__ x1, const float* __restrict__ x2,
                                                     const tat_bf16* __restrict__ w, const float* __restrict__ bias,
                                                     tat_bf16* __restrict__ h) {
  TAT_GRID_DEPENDENCY();
  constexpr int KV = 9 * CIN;
  __shared__ __align__(16) unsigned short xs[CIN * XH * XW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  unsigned bw[2][4][2];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int k = ks * 16 + hf * 8 + 2 * t, n = nt * 8 + g;
        const unsigned lo = k < KV ? w[k * C + n] : 0u, hi = k + 1 < KV ? w[(k + 1) * C + n] : 0u;
        bw[ks][nt][hf] = lo | (hi << 16);
      }
  // halo offsets of the thread's A columns k = 16 ks + {2t, 2t+1, 2t+8, 2t+9}; -1 past K
  int aoff[2][4];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = ks * 16 + 2 * t + (j & 1) + (j >> 1) * 8, tap = k / CIN;
      aoff[ks][j] = k < KV ? (k % CIN) * XH * XW + (tap / 3) * XW + tap % 3 + warp * XW : -1;
    }
  float xv[kXPer];
  tile_loop(
      B, H, W, nullptr, 0, [](int, int, int, int) {},
      [&](int b, int y0, int x0c) { x_prefetch<CIN>(xv, x0, x1, x2, b, y0, x0c, H, W); },
      [&] {
#pragma unroll
        for (int k = 0; k < kXPer; ++k) {
          const int e = threadIdx.x + 256 * k;
          if (e < CIN * XH * XW) xs[e] = tobf(xv[k]);
        }
      },
      [&](int b, int y0, int x0c, int) {
        float acc[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[nt][k] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          auto ld = [&](int j, int px) -> unsigned { return aoff[ks][j] < 0 ? 0u : (unsigned)xs[aoff[ks][j] + px]; };
          const unsigned a[4] = {ld(0, g) | (ld(1, g) << 16), ld(0, g + 8) | (ld(1, g + 8) << 16),
                                 ld(2, g) | (ld(3, g) << 16), ld(2, g + 8) | (ld(3, g + 8) << 16)};
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[nt], a, bw[ks][nt]);
        }
        const int y = y0 + warp;
        if (y >= H) return;
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int x = x0c + g + 8 * hf;
          if (x >= W) continue;
          tat_bf16* dst = h + (((long long)b * H + y) * W + x) * C;
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const int co = nt * 8 + 2 * t;
            const float v0 = fmaxf(acc[nt][2 * hf] + bias[co], 0.f), v1 = fmaxf(acc[nt][2 * hf + 1] + bias[co + 1], 0.f);
            *reinterpret_cast<unsigned*>(dst + co) = (unsigned)tobf(v0) | ((unsigned)tobf(v1) << 16);
          }
        }
      });
}

// Layout of k_conv_in_bwd's dynamic shared memory: alignment slack; two slots of the g
// halo (and, with MASK, the h halo), a region that afterwards holds the per-warp weight-
// gradient sums; the per-tap sums z[9 CIN][ZP] of the data gradient; two BF16 copies of the
// x halo (the second shifted by one column, so that every pixel pair is a 4-byte word in one
// of them); two mbarriers.
template <int CIN, bool MASK>
struct InBwdSmem {
  static constexpr int STAGE = (MASK ? 2 : 1) * HALO_SLOT;
  static constexpr int NTW = (9 * CIN + 1 + 7) / 8;  // n-tiles of the weight-gradient GEMM (with the ones column)
  static constexpr int NTZ = (9 * CIN + 7) / 8;      // n-tiles of the per-tap sums
  static constexpr int RED = 8 * NTW * 8 * C * 4;
  static constexpr int REGION = 2 * STAGE > RED ? 2 * STAGE : RED;
  static constexpr int XCOPY = CIN * XH * XP;
  static constexpr int ZS = REGION, XS = ZS + 9 * CIN * ZP * 4, BAR = XS + 2 * XCOPY * 2;
  static constexpr size_t BYTES = 1024 + BAR + 2 * sizeof(uint64_t);
};

// Backward of the in layer in one pass over the tiles of G' = g_h * [h > 0] (with MASK;
// without it g_h arrives masked, as tat_conv_mid_bwd_data with h_in writes it):
//   DATA : gx_c(p) = sum_{tap, co} G'(p - tap)[co] w[tap][c][co]   (A = shifted G', N = 8 >= CIN)
//   WGRAD: dW[tap * CIN + c][co] = sum_p G'(p)[co] x_c(p + tap), db[co] = sum_p G'(p)[co]
//          (A = G'^T by ldmatrix.trans, B = x pairs, plus a column of ones for db), per-CTA
//          partials [9 CIN + 1][32].
// DATA and WGRAD are the bits 1 and 2 of `parts` (uniform branches).
template <int CIN, bool MASK>
__global__ void __launch_bounds__(256, 2) k_conv_in_bwd(int B, int H, int W, const __grid_constant__ CUtensorMap map_g,
                                                        const __grid_constant__ CUtensorMap map_h,
                                                        const float* __restrict__ x0, const float* __restrict__ x1,
                                                        const float* __restrict__ x2, const tat_bf16* __restrict__ w,
                                                        float* gx0, float* gx1, float* gx2, int accumulate, int parts,
                                                        float* __restrict__ partial) {
  TAT_GRID_DEPENDENCY();
  using L = InBwdSmem<CIN, MASK>;
  constexpr int KV = 9 * CIN, NTW = L::NTW, STAGE = L::STAGE, XCOPY = L::XCOPY;
  const bool DATA = parts & 1, WGRAD = parts & 2;
  extern __shared__ unsigned char dsm[];
  unsigned char* sm = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
  float* zs = reinterpret_cast<float*>(sm + L::ZS);
  unsigned short* xs = reinterpret_cast<unsigned short*>(sm + L::XS);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // B of the per-tap sums: B[k = co][n = tap CIN + c] = w[8 - tap][c][co] (the flipped kernel)
  unsigned bz[2][L::NTZ][2];
#pragma unroll
  for (int kc = 0; kc < 2; ++kc)
#pragma unroll
    for (int nt = 0; nt < L::NTZ; ++nt)
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int n = 8 * nt + g, co = 16 * kc + 8 * hf + 2 * t;
        const int tap = n / CIN, c = n % CIN;
        bz[kc][nt][hf] = DATA && n < KV ? (unsigned)w[((8 - tap) * CIN + c) * C + co] |
                                              ((unsigned)w[((8 - tap) * CIN + c) * C + co + 1] << 16)
                                        : 0u;
      }
  // B of the weight gradient: per n-tile the word offset of the thread's x pair (column n = 8 nt + g)
  int boff[NTW];
  unsigned bconst[NTW];
#pragma unroll
  for (int nt = 0; nt < NTW; ++nt) {
    const int n = nt * 8 + g;
    boff[nt] = -1;
    bconst[nt] = n == KV ? 0x3f803f80u : 0u;  // (1, 1) in BF16 for the bias column
    if (n < KV) {
      const int tap = n / CIN, c = n % CIN, dy = tap / 3, dx = tap % 3;
      boff[nt] = dx == 1 ? XCOPY + c * XH * XP + (warp + dy) * XP + 2 * t : c * XH * XP + (warp + dy) * XP + 2 * t + dx;
    }
  }
  init_bars(bar);
  __syncthreads();
  float accw[2][NTW][4];
#pragma unroll
  for (int mh = 0; mh < 2; ++mh)
#pragma unroll
    for (int nt = 0; nt < NTW; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) accw[mh][nt][k] = 0.f;
  float xv[kXPer];
  const bool ok = tile_loop(
      B, H, W, bar, (MASK ? 2 : 1) * HALO_BYTES,
      [&](int b, int y0, int x0c, int s) {
        tma_load_4d(sm + s * STAGE, &map_g, 0, x0c - 1, y0 - 1, b, &bar[s]);
        if (MASK) tma_load_4d(sm + s * STAGE + HALO_SLOT, &map_h, 0, x0c - 1, y0 - 1, b, &bar[s]);
      },
      [&](int b, int y0, int x0c) {
        if (WGRAD) x_prefetch<CIN>(xv, x0, x1, x2, b, y0, x0c, H, W);
      },
      [&] {
        if (WGRAD)
#pragma unroll
          for (int k = 0; k < kXPer; ++k) {
            const int e = threadIdx.x + 256 * k;
            if (e < CIN * XH * XW) {
              const int c = e / (XH * XW), r = (e / XW) % XH, j = e % XW;
              const unsigned short v = tobf(xv[k]);
              xs[c * XH * XP + r * XP + j] = v;
              if (j > 0) xs[XCOPY + c * XH * XP + r * XP + j - 1] = v;
            }
          }
      },
      [&](int b, int y0, int x0c, int s) {
        const unsigned char* gt = sm + s * STAGE;
        const unsigned char* ht = gt + HALO_SLOT;
        const int m = lane >> 3;
        if (DATA) {
          // per-tap sums z[tap CIN + c](q) = sum_co G'(q)[co] w[8 - tap][c][co] of every halo
          // pixel q (12 m-tiles of 16; the last one partly past the halo, inside the slot) ...
          for (int mt = warp; mt < 12; mt += 8) {
            float acc[L::NTZ][4];
#pragma unroll
            for (int nt = 0; nt < L::NTZ; ++nt)
#pragma unroll
              for (int k = 0; k < 4; ++k) acc[nt][k] = 0.f;
            const int pa = 16 * mt + (m & 1) * 8 + (lane & 7);
#pragma unroll
            for (int kc = 0; kc < 2; ++kc) {
              unsigned a[4];
              ldsm_x4(a, swz(gt, pa, 2 * kc + (m >> 1)));
              if (MASK) {
                unsigned mk[4];
                ldsm_x4(mk, swz(ht, pa, 2 * kc + (m >> 1)));
#pragma unroll
                for (int j = 0; j < 4; ++j) a[j] = relu_masked(a[j], mk[j]);
              }
#pragma unroll
              for (int nt = 0; nt < L::NTZ; ++nt) mma_bf16(acc[nt], a, bz[kc][nt]);
            }
            const int q = 16 * mt + g;
#pragma unroll
            for (int nt = 0; nt < L::NTZ; ++nt)
#pragma unroll
              for (int j = 0; j < 2; ++j) {
                const int n = 8 * nt + 2 * t + j;
                if (n < KV) {
                  zs[n * ZP + q] = acc[nt][j];
                  zs[n * ZP + q + 8] = acc[nt][2 + j];
                }
              }
          }
          __syncthreads();
          // ... then gx_c(p) = sum_tap z[tap CIN + c](p + tap), a 9-point stencil
          if (threadIdx.x < TY * TX) {
            const int r = threadIdx.x >> 4, cc = threadIdx.x & 15;
            const int y = y0 + r, x = x0c + cc;
            if (y < H && x < W) {
              const long long pix = ((long long)b * H + y) * W + x;
#pragma unroll
              for (int c = 0; c < CIN; ++c) {
                float* gx = c == 0 ? gx0 : (c == 1 ? gx1 : gx2);
                if (gx == nullptr) continue;
                float v = 0.f;
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) v += zs[(tap * CIN + c) * ZP + (r + tap / 3) * XW + cc + tap % 3];
                gx[pix] = (((accumulate >> c) & 1) ? gx[pix] : 0.f) + v;
              }
            }
          }
        }
        if (WGRAD) {
          unsigned a[2][4];
#pragma unroll
          for (int mh = 0; mh < 2; ++mh) {
            // A = G'^T (co x pixel): matrices (co 0-7, px 0-7), (co 8-15, px 0-7), (co 0-7, px 8-15), (co 8-15, px 8-15)
            const int p = (warp + 1) * XW + 1 + (m >> 1) * 8 + (lane & 7);
            ldsm_x4_trans(a[mh], swz(gt, p, 2 * mh + (m & 1)));
            if (MASK) {
              unsigned mk[4];
              ldsm_x4_trans(mk, swz(ht, p, 2 * mh + (m & 1)));
#pragma unroll
              for (int j = 0; j < 4; ++j) a[mh][j] = relu_masked(a[mh][j], mk[j]);
            }
          }
#pragma unroll
          for (int nt = 0; nt < NTW; ++nt) {
            unsigned bb[2] = {bconst[nt], bconst[nt]};
            if (boff[nt] >= 0) {
              bb[0] = *reinterpret_cast<const unsigned*>(xs + boff[nt]);
              bb[1] = *reinterpret_cast<const unsigned*>(xs + boff[nt] + 8);
            }
            mma_bf16(accw[0][nt], a[0], bb);
            mma_bf16(accw[1][nt], a[1], bb);
          }
        }
      });
  if (!WGRAD || !ok) return;
  // per-warp sums [warp][n][co] in the (now idle) tile slots, then a fixed-order sum over the warps
  constexpr int NW = (KV + 1) * C;
  float* red = reinterpret_cast<float*>(sm);
#pragma unroll
  for (int mh = 0; mh < 2; ++mh)
#pragma unroll
    for (int nt = 0; nt < NTW; ++nt) {
      const int co = mh * 16 + g, n = nt * 8 + 2 * t;
      float* r = red + warp * NTW * 8 * C;
      r[n * C + co] = accw[mh][nt][0];
      r[(n + 1) * C + co] = accw[mh][nt][1];
      r[n * C + co + 8] = accw[mh][nt][2];
      r[(n + 1) * C + co + 8] = accw[mh][nt][3];
    }
  __syncthreads();
  for (int o = threadIdx.x; o < NW; o += blockDim.x) {
    float sum = 0.f;
#pragma unroll
    for (int wp = 0; wp < 8; ++wp) sum += red[wp * NTW * 8 * C + o];
    partial[(size_t)blockIdx.x * NW + o] = sum;
  }
}

// Dynamic shared memory of the out-layer kernels: alignment slack, two slots of h halos,
// the per-tap sums z[9][ZP] (forward) or the hi / lo x 2-copy halo of g_out (backward), two
// mbarriers.
constexpr size_t out_fwd_smem_bytes() { return 1024 + 2 * HALO_SLOT + 9 * ZP * 4 + 2 * sizeof(uint64_t); }
constexpr size_t out_bwd_smem_bytes() { return 1024 + 2 * HALO_SLOT + 4 * XH * XP * 2 + 2 * sizeof(uint64_t); }

// out = residual + b + conv_out(h), in two steps per tile.  First the per-tap channel sums
// z[tap](q) = sum_ci w[tap][ci] h(q)[ci] of every halo pixel q: a GEMM with M = the halo's
// pixels (12 m-tiles of 16, the last one partly past the halo, inside the slot), N = 16
// (taps, 9 used), K = 32 channels, A by ldmatrix from the swizzled halo -- each halo value
// is read once.  Then out(p) = sum_tap z[tap](p + tap), a 9-point stencil on z in shared
// memory.
__global__ void __launch_bounds__(256) k_conv_out_fwd(int B, int H, int W, const __grid_constant__ CUtensorMap map_h,
                                                      const tat_bf16* __restrict__ w, const float* __restrict__ bias,
                                                      const float* residual, float* out) {
  TAT_GRID_DEPENDENCY();
  extern __shared__ unsigned char dsm[];
  unsigned char* sm = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
  float* zs = reinterpret_cast<float*>(sm + 2 * HALO_SLOT);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * HALO_SLOT + 9 * ZP * 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // B[k = ci][n = tap] fragments of the two k-steps and two n-tiles (taps 9..15 zero)
  unsigned bq[2][2][2];
#pragma unroll
  for (int kc = 0; kc < 2; ++kc)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int hf = 0; hf < 2; ++hf) {
        const int tap = 8 * nt + g, ci = 16 * kc + 8 * hf + 2 * t;
        bq[kc][nt][hf] = tap < 9 ? (unsigned)w[tap * C + ci] | ((unsigned)w[tap * C + ci + 1] << 16) : 0u;
      }
  init_bars(bar);
  __syncthreads();
  const float b0 = bias[0];
  const int m = lane >> 3;
  tile_loop(
      B, H, W, bar, HALO_BYTES,
      [&](int b, int y0, int x0c, int s) { tma_load_4d(sm + s * HALO_SLOT, &map_h, 0, x0c - 1, y0 - 1, b, &bar[s]); },
      [](int, int, int) {}, [] {},
      [&](int b, int y0, int x0c, int s) {
        const unsigned char* ht = sm + s * HALO_SLOT;
        for (int mt = warp; mt < 12; mt += 8) {
          float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
          for (int kc = 0; kc < 2; ++kc) {
            unsigned a[4];
            ldsm_x4(a, swz(ht, 16 * mt + (m & 1) * 8 + (lane & 7), 2 * kc + (m >> 1)));
            mma_bf16(acc[0], a, bq[kc][0]);
            mma_bf16(acc[1], a, bq[kc][1]);
          }
          const int q = 16 * mt + g;
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            const int tap = 8 * nt + 2 * t;
            if (tap < 9) {
              zs[tap * ZP + q] = acc[nt][0];
              zs[tap * ZP + q + 8] = acc[nt][2];
            }
            if (tap + 1 < 9) {
              zs[(tap + 1) * ZP + q] = acc[nt][1];
              zs[(tap + 1) * ZP + q + 8] = acc[nt][3];
            }
          }
        }
        __syncthreads();
        const int r = threadIdx.x >> 4, c = threadIdx.x & 15;  // 256 threads = the 8 x 16 outputs, twice
        if (threadIdx.x < TY * TX) {
          const int y = y0 + r, x = x0c + c;
          if (y < H && x < W) {
            float v = 0.f;
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) v += zs[tap * ZP + (r + tap / 3) * XW + c + tap % 3];
            const long long pix = ((long long)b * H + y) * W + x;
            out[pix] = residual[pix] + b0 + v;
          }
        }
      });
}

// Backward of the out layer in one pass (g = g_out split as hi + lo):
//   g_h(p)[ci] = sum_tap g(p - tap) w[tap][ci]           (A[pixel][tap] gathered, B = w, N = 32),
//                times [h(p)[ci] > 0] with MASK (the gradient of the mid layer's pre-activation)
//   dW[tap][ci] = sum_q h(q)[ci] g(q - tap), db = sum g   (A = h^T by ldmatrix.trans, B = g pairs,
//                                                          n = part * 9 + tap), per-CTA partials [289].
template <bool MASK>
__global__ void __launch_bounds__(256, 2) k_conv_out_bwd(int B, int H, int W, const __grid_constant__ CUtensorMap map_h,
                                                         const float* __restrict__ gout, const tat_bf16* __restrict__ w,
                                                         tat_bf16* __restrict__ gh, float* __restrict__ partial) {
  TAT_GRID_DEPENDENCY();
  constexpr int PART = 2 * XH * XP, CPY = XH * XP;  // gs[part][copy][XH][XP]
  extern __shared__ unsigned char dsm[];
  unsigned char* sm = dsm + ((1024u - (smem_u32(dsm) & 1023u)) & 1023u);
  unsigned short* gs = reinterpret_cast<unsigned short*>(sm + 2 * HALO_SLOT);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * HALO_SLOT + 4 * XH * XP * 2);
  __shared__ float dbred[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // B of g_h: w[k = tap][n = ci], K = 16 (taps 9..15 zero)
  unsigned bo[4][2];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int n = nt * 8 + g, k = 2 * t;
    bo[nt][0] = (unsigned)w[k * C + n] | ((unsigned)w[(k + 1) * C + n] << 16);
    bo[nt][1] = k + 8 < 9 ? (unsigned)w[(k + 8) * C + n] : 0u;
  }
  // A of g_h: halo offsets of the taps k = 2t, 2t+1, 2t+8, 2t+9 (g(p - tap) sits at halo row
  // r + 2 - tap / 3, column j + 2 - tap % 3); -1 for k >= 9
  int goff[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = 2 * t + (j & 1) + (j >> 1) * 8;
    goff[j] = k < 9 ? (warp + 2 - k / 3) * XP + 2 - k % 3 : -1;
  }
  // B of dW: word offset of the thread's g pair for column n = 8 nt + g (part n / 9, tap n % 9)
  int boff[3];
#pragma unroll
  for (int nt = 0; nt < 3; ++nt) {
    const int n = nt * 8 + g;
    boff[nt] = -1;
    if (n < 18) {
      const int part = n / 9, tap = n % 9, dxo = 2 - tap % 3;
      boff[nt] = part * PART + (warp + 2 - tap / 3) * XP + (dxo == 1 ? CPY + 2 * t : 2 * t + dxo);
    }
  }
  init_bars(bar);
  __syncthreads();
  float accw[2][3][4];
#pragma unroll
  for (int mh = 0; mh < 2; ++mh)
#pragma unroll
    for (int nt = 0; nt < 3; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) accw[mh][nt][k] = 0.f;
  float gv = 0.f, dbacc = 0.f;
  int gr = 0, gj = 0;
  const bool ok = tile_loop(
      B, H, W, bar, HALO_BYTES,
      [&](int b, int y0, int x0c, int s) { tma_load_4d(sm + s * HALO_SLOT, &map_h, 0, x0c - 1, y0 - 1, b, &bar[s]); },
      [&](int b, int y0, int x0c) {
        gv = 0.f;
        gr = threadIdx.x / XW;
        gj = threadIdx.x % XW;
        if (threadIdx.x < XH * XW) {
          const int yy = y0 - 1 + gr, xx = x0c - 1 + gj;
          if (yy >= 0 && yy < H && xx >= 0 && xx < W) gv = gout[((long long)b * H + yy) * W + xx];
        }
      },
      [&] {
        if (threadIdx.x < XH * XW) {
          const unsigned short hi = tobf(gv), lo = tobf(gv - bf(hi));
          gs[gr * XP + gj] = hi;
          gs[PART + gr * XP + gj] = lo;
          if (gj > 0) {
            gs[CPY + gr * XP + gj - 1] = hi;
            gs[PART + CPY + gr * XP + gj - 1] = lo;
          }
          if (gr >= 1 && gr <= TY && gj >= 1 && gj <= TX) dbacc += gv;
        }
      },
      [&](int b, int y0, int x0c, int s) {
        const unsigned char* ht = sm + s * HALO_SLOT;
        const int m = lane >> 3;
        // g_h
        {
          float acc[4][4];
#pragma unroll
          for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[nt][k] = 0.f;
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            auto ld = [&](int j, int px) -> unsigned {
              return goff[j] < 0 ? 0u : (unsigned)gs[part * PART + goff[j] + px];
            };
            const unsigned a[4] = {ld(0, g) | (ld(1, g) << 16), ld(0, g + 8) | (ld(1, g + 8) << 16),
                                   ld(2, g) | (ld(3, g) << 16), ld(2, g + 8) | (ld(3, g + 8) << 16)};
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[nt], a, bo[nt]);
          }
          const int y = y0 + warp;
          if (y < H) {
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
              const int x = x0c + g + 8 * hf;
              if (x >= W) continue;
              tat_bf16* dst = gh + (((long long)b * H + y) * W + x) * C;
              const int p = (warp + 1) * XW + g + 8 * hf + 1;  // this pixel in the staged h halo
#pragma unroll
              for (int nt = 0; nt < 4; ++nt) {
                unsigned v = (unsigned)tobf(acc[nt][2 * hf]) | ((unsigned)tobf(acc[nt][2 * hf + 1]) << 16);
                if (MASK)
                  v = relu_masked(v, *reinterpret_cast<const unsigned*>(swz(ht, p, nt) + 4 * t));
                *reinterpret_cast<unsigned*>(dst + nt * 8 + 2 * t) = v;
              }
            }
          }
        }
        // dW
        unsigned a[2][4];
#pragma unroll
        for (int mh = 0; mh < 2; ++mh) {
          const int p = (warp + 1) * XW + 1 + (m >> 1) * 8 + (lane & 7);
          ldsm_x4_trans(a[mh], swz(ht, p, 2 * mh + (m & 1)));
        }
#pragma unroll
        for (int nt = 0; nt < 3; ++nt) {
          unsigned bb[2] = {0u, 0u};
          if (boff[nt] >= 0) {
            bb[0] = *reinterpret_cast<const unsigned*>(gs + boff[nt]);
            bb[1] = *reinterpret_cast<const unsigned*>(gs + boff[nt] + 8);
          }
          mma_bf16(accw[0][nt], a[0], bb);
          mma_bf16(accw[1][nt], a[1], bb);
        }
      });
  if (!ok) return;
  float* red = reinterpret_cast<float*>(sm);  // [warp][24][32] in the idle tile slots
#pragma unroll
  for (int mh = 0; mh < 2; ++mh)
#pragma unroll
    for (int nt = 0; nt < 3; ++nt) {
      const int ci = mh * 16 + g, n = nt * 8 + 2 * t;
      float* r = red + warp * 24 * C;
      r[n * C + ci] = accw[mh][nt][0];
      r[(n + 1) * C + ci] = accw[mh][nt][1];
      r[n * C + ci + 8] = accw[mh][nt][2];
      r[(n + 1) * C + ci + 8] = accw[mh][nt][3];
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dbacc += __shfl_xor_sync(0xffffffffu, dbacc, o);
  if (lane == 0) dbred[warp] = dbacc;
  __syncthreads();
  constexpr int NW = 9 * C + 1;
  for (int o = threadIdx.x; o < NW; o += blockDim.x) {
    float sum = 0.f;
    if (o < 9 * C) {
#pragma unroll
      for (int wp = 0; wp < 8; ++wp) sum += red[wp * 24 * C + o] + red[wp * 24 * C + 9 * C + o];
    } else {
#pragma unroll
      for (int wp = 0; wp < 8; ++wp) sum += dbred[wp];
    }
    partial[(size_t)blockIdx.x * NW + o] = sum;
  }
}

// ------------------------------------------------------------------ optimizer and loss

__global__ void k_adam(long long n, float lr, float b1, float b2, float eps, float c1, float c2, float* p,
                       const float* __restrict__ g, float* m, float* v, tat_bf16* wb) {
  TAT_GRID_DEPENDENCY();
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
  TAT_GRID_DEPENDENCY();
  GRID_STRIDE(i, n) out[i] = value;
}

__global__ void k_to_bf16(long long n, const float* __restrict__ x, tat_bf16* out) {
  TAT_GRID_DEPENDENCY();
  GRID_STRIDE(i, n) out[i] = tobf(x[i]);
}

__global__ void k_mse(long long n, const float* __restrict__ a, const float* __restrict__ b, float scale, float* grad,
                      float* loss) {
  TAT_GRID_DEPENDENCY();
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

bool bad_sizes(int batch, int H, int W) {
  return batch < 1 || H < 1 || W < 1 || (long long)batch * H * W >= (1LL << 31);  // tiles are counted in 32 bits
}

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

// Raises the dynamic shared-memory limit of `Kern` to `bytes` once per device.
template <auto Kern>
bool smem_attr(size_t bytes) {
  static int done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return false;
  }
  if (!done[dev]) {
    if (cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    done[dev] = 1;
  }
  return true;
}

bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; }

// Tensor map of a [batch][H][W][32] BF16 activation for the tcgen05 kernel: the 18 x 10
// halo of 32 channels in one box, 64-byte swizzle (the MMA's swizzled K-major layout).
bool halo_tc_map(CUtensorMap* m, const tat_bf16* base, int batch, int H, int W) {
  const EncodeTiled fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)batch};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
  const cuuint32_t box[4] = {(cuuint32_t)C, (cuuint32_t)tc::HX, (cuuint32_t)tc::HY, 1};
  const cuuint32_t estride[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<tat_bf16*>(base), dims, strides, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of the tcgen05 kernel's output: one 16 x 8-pixel tile of 32 channels per box
// (the shared-memory staging tile [y][x][32], no swizzle).
bool tile_out_map(CUtensorMap* m, tat_bf16* base, int batch, int H, int W) {
  const EncodeTiled fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)batch};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
  const cuuint32_t box[4] = {(cuuint32_t)C, (cuuint32_t)tc::TX, (cuuint32_t)tc::TY, 1};
  const cuuint32_t estride[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool BWD, bool OMASK>
tat_status launch_mid_tc(int batch, int H, int W, const CUtensorMap& m8, const tat_bf16* w, const float* b,
                         const tat_bf16* omask, tat_bf16* out, cudaStream_t s, const char* what) {
  constexpr size_t smem = tc::SMEM;
  if (!smem_attr<k_conv_mid_tc<BWD, OMASK>>(smem)) return TAT_ERR_CUDA;
  CUtensorMap mo;
  if (!tile_out_map(&mo, out, batch, H, W)) {
    fprintf(stderr, "%s: tensor map encoding failed\n", what);
    return TAT_ERR_CUDA;
  }
  const long long tiles = (long long)batch * ((H + tc::TY - 1) / tc::TY) * ((W + tc::TX - 1) / tc::TX);
  const int ctas = (int)(tiles < tc::CTAS * 152 ? tiles : tc::CTAS * 152);  // persistent: all resident
  tat::pdl_launch(true, k_conv_mid_tc<BWD, OMASK>, ctas, 192, smem, s, batch, H, W, m8, mo, w, b, omask);
  return launched(what);
}

template <bool BWD, bool MASK, bool OMASK>
tat_status launch_mid(int batch, int H, int W, const tat_bf16* in, const tat_bf16* mask, const tat_bf16* omask,
                      const tat_bf16* w, const float* b, tat_bf16* out, cudaStream_t s, const char* what) {
  if (misaligned(in) || misaligned(mask) || misaligned(omask)) return TAT_ERR_INVALID_ARG;
  CUtensorMap mi, mm, mo;
  if (!halo_map(&mi, in, batch, H, W) || !halo_map(&mm, MASK ? mask : in, batch, H, W) ||
      !halo_map(&mo, OMASK ? omask : in, batch, H, W)) {
    fprintf(stderr, "%s: tensor map encoding failed\n", what);
    return TAT_ERR_CUDA;
  }
  constexpr size_t smem = mid_smem_bytes<1 + MASK + OMASK>();
  if (!smem_attr<k_conv_mid<BWD, MASK, OMASK>>(smem)) return TAT_ERR_CUDA;
  tat::pdl_launch(true, k_conv_mid<BWD, MASK, OMASK>, mid_ctas(batch, H, W), 256, smem, s, batch, H, W, mi, mm, mo, w, b, out);
  return launched(what);
}

// CTAs of the persistent thin-layer kernels: up to `per_sm` per SM, never more than the tiles.
int thin_ctas(int batch, int H, int W, int per_sm) {
  const long long tiles = (long long)batch * ((H + TY - 1) / TY) * ((W + TX - 1) / TX);
  return (int)(tiles < per_sm * 152LL ? tiles : per_sm * 152LL);
}

template <int CIN, bool MASK>
tat_status launch_in_bwd(int batch, int H, int W, const CUtensorMap& mg, const CUtensorMap& mh, const float* x0,
                         const float* x1, const float* x2, const tat_bf16* w, float* gx0, float* gx1, float* gx2,
                         int accumulate, int parts, float* scratch, int ctas, cudaStream_t s) {
  constexpr size_t smem = InBwdSmem<CIN, MASK>::BYTES;
  if (!smem_attr<k_conv_in_bwd<CIN, MASK>>(smem)) return TAT_ERR_CUDA;
  tat::pdl_launch(true, k_conv_in_bwd<CIN, MASK>, ctas, 256, smem, s, batch, H, W, mg, mh, x0, x1, x2, w, gx0, gx1, gx2, accumulate, parts, scratch);
  return launched("tat_conv_in_bwd");
}

template <int CIN>
tat_status in_bwd(int batch, int H, int W, const float* x0, const float* x1, const float* x2, const tat_bf16* g_h,
                  const tat_bf16* h, const tat_bf16* w, float* gx0, float* gx1, float* gx2, int accumulate,
                  float* scratch, size_t scratch_floats, float* gw, float* gb, cudaStream_t s) {
  const bool data = gx0 || gx1 || gx2, wgrad = gw != nullptr;
  if (!data && !wgrad) return TAT_OK;
  const int ctas = thin_ctas(batch, H, W, 2);
  const int nw = (9 * CIN + 1) * C;
  if (wgrad && scratch_floats < (size_t)ctas * nw) return TAT_ERR_INVALID_ARG;
  CUtensorMap mg, mh;
  if (!halo_map(&mg, g_h, batch, H, W) || !halo_map(&mh, h ? h : g_h, batch, H, W)) {
    fprintf(stderr, "tat_conv_in_bwd: tensor map encoding failed\n");
    return TAT_ERR_CUDA;
  }
  const int parts = (data ? 1 : 0) | (wgrad ? 2 : 0);
  const tat_status st =
      h ? launch_in_bwd<CIN, true>(batch, H, W, mg, mh, x0, x1, x2, w, gx0, gx1, gx2, accumulate, parts, scratch, ctas, s)
        : launch_in_bwd<CIN, false>(batch, H, W, mg, mh, x0, x1, x2, w, gx0, gx1, gx2, accumulate, parts, scratch, ctas,
                                    s);
  if (st != TAT_OK || !wgrad) return st;
  tat::pdl_launch(true, k_reduce_partials, (nw + 31) / 32, 1024, 0, s, ctas, 9 * CIN * C, C, scratch, gw, gb);
  return launched("tat_conv_in_bwd");
}

// Tensor maps of k_conv_mid_wgrad_tc: 32 channels x `bx` x `by` pixels, 64-byte swizzle.
bool wgrad_tc_map(CUtensorMap* m, const tat_bf16* base, int batch, int H, int W, int bx, int by) {
  const EncodeTiled fn = encoder();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)batch};
  const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
  const cuuint32_t box[4] = {(cuuint32_t)C, (cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t estride[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<tat_bf16*>(base), dims, strides, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int wgrad_ctas(int batch, int H, int W) {
  const long long tiles = (long long)batch * ((H + TY - 1) / TY) * ((W + TX - 1) / TX);
  return (int)(tiles < kMaxCtas ? tiles : kMaxCtas);
}

}  // namespace

extern "C" {

size_t tat_lpd_scratch_floats(int batch, int H, int W) {
  if (bad_sizes(batch, H, W)) return 0;
  return (size_t)kMaxCtas * (9 * C * C + C);  // the largest of the per-CTA partial sets
}

tat_status tat_conv_in_fwd(int batch, int H, int W, int cin, const float* x0, const float* x1, const float* x2,
                           const tat_bf16* w, const float* b, tat_bf16* h, tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || (cin != 2 && cin != 3) || !x0 || !x1 || (cin == 3 && !x2) || !w || !b || !h)
    return TAT_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ctas = thin_ctas(batch, H, W, 3);
  if (cin == 2) tat::pdl_launch(true, k_conv_in_fwd<2>, ctas, 256, 0, s, batch, H, W, x0, x1, nullptr, w, b, h);
  else tat::pdl_launch(true, k_conv_in_fwd<3>, ctas, 256, 0, s, batch, H, W, x0, x1, x2, w, b, h);
  return launched("tat_conv_in_fwd");
}

tat_status tat_conv_in_bwd(int batch, int H, int W, int cin, const float* x0, const float* x1, const float* x2,
                           const tat_bf16* g_h, const tat_bf16* h, const tat_bf16* w, float* gx0, float* gx1,
                           float* gx2, int accumulate, float* scratch, size_t scratch_floats, float* gw, float* gb,
                           tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || (cin != 2 && cin != 3) || !g_h || misaligned(g_h) || misaligned(h))
    return TAT_ERR_INVALID_ARG;
  if ((gx0 || gx1 || gx2) && !w) return TAT_ERR_INVALID_ARG;
  if (gw && (!x0 || !x1 || (cin == 3 && !x2) || !scratch || !gb)) return TAT_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cin == 2)
    return in_bwd<2>(batch, H, W, x0, x1, nullptr, g_h, h, w, gx0, gx1, nullptr, accumulate, scratch, scratch_floats,
                     gw, gb, s);
  return in_bwd<3>(batch, H, W, x0, x1, x2, g_h, h, w, gx0, gx1, gx2, accumulate, scratch, scratch_floats, gw, gb, s);
}

tat_status tat_conv_in_bwd_data(int batch, int H, int W, int cin, const tat_bf16* g_h, const tat_bf16* h,
                                const tat_bf16* w, float* gx0, float* gx1, float* gx2, int accumulate,
                                tat_stream_t stream) {
  return tat_conv_in_bwd(batch, H, W, cin, nullptr, nullptr, nullptr, g_h, h, w, gx0, gx1, cin == 3 ? gx2 : nullptr,
                         accumulate, nullptr, 0, nullptr, nullptr, stream);
}

tat_status tat_conv_in_bwd_weights(int batch, int H, int W, int cin, const float* x0, const float* x1,
                                   const float* x2, const tat_bf16* g_h, const tat_bf16* h, float* scratch,
                                   size_t scratch_floats, float* gw, float* gb, tat_stream_t stream) {
  if (!gw) return TAT_ERR_INVALID_ARG;
  return tat_conv_in_bwd(batch, H, W, cin, x0, x1, x2, g_h, h, nullptr, nullptr, nullptr, nullptr, 0, scratch,
                         scratch_floats, gw, gb, stream);
}

tat_status tat_conv_mid_fwd(int batch, int H, int W, const tat_bf16* h_in, const tat_bf16* w, const float* b,
                            tat_bf16* h_out, tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || !h_in || !w || !b || !h_out || misaligned(h_in) || misaligned(h_out) ||
      misaligned(w))
    return TAT_ERR_INVALID_ARG;
  CUtensorMap m8;
  if (!halo_tc_map(&m8, h_in, batch, H, W)) {
    fprintf(stderr, "tat_conv_mid_fwd: tensor map encoding failed\n");
    return TAT_ERR_CUDA;
  }
  return launch_mid_tc<false, false>(batch, H, W, m8, w, b, nullptr, h_out, static_cast<cudaStream_t>(stream),
                                     "tat_conv_mid_fwd");
}

tat_status tat_conv_mid_bwd_data(int batch, int H, int W, const tat_bf16* g_out, const tat_bf16* h_out,
                                 const tat_bf16* w, const tat_bf16* h_in, tat_bf16* g_in, tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || !g_out || !w || !g_in || misaligned(w)) return TAT_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  const char* what = "tat_conv_mid_bwd_data";
  if (h_out && h_in) return launch_mid<true, true, true>(batch, H, W, g_out, h_out, h_in, w, nullptr, g_in, s, what);
  if (h_out) return launch_mid<true, true, false>(batch, H, W, g_out, h_out, nullptr, w, nullptr, g_in, s, what);
  // an already masked gradient: the tcgen05 kernel
  if (misaligned(g_out) || misaligned(h_in) || misaligned(g_in)) return TAT_ERR_INVALID_ARG;
  CUtensorMap m8;
  if (!halo_tc_map(&m8, g_out, batch, H, W)) {
    fprintf(stderr, "%s: tensor map encoding failed\n", what);
    return TAT_ERR_CUDA;
  }
  if (h_in) return launch_mid_tc<true, true>(batch, H, W, m8, w, nullptr, h_in, g_in, s, what);
  return launch_mid_tc<true, false>(batch, H, W, m8, w, nullptr, nullptr, g_in, s, what);
}

tat_status tat_lpd_timeout_probe(int tries, int* gave_up, tat_stream_t stream) {
  if (tries < 1 || tries > (1 << 20) || !gave_up) return TAT_ERR_INVALID_ARG;
  k_wait_probe<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(tries, gave_up);
  return launched("tat_lpd_timeout_probe");
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
  if (bad_sizes(batch, H, W) || !h_in || !g_out || !scratch || !gw || !gb || misaligned(h_in) ||
      misaligned(g_out) || misaligned(h_out))
    return TAT_ERR_INVALID_ARG;
  const int ctas = wgrad_ctas(batch, H, W);
  const int nw = 9 * C * C + C;
  if (scratch_floats < (size_t)ctas * nw) return TAT_ERR_INVALID_ARG;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  CUtensorMap mi, mg, mh;
  if (!halo_map(&mi, h_in, batch, H, W) || !halo_map(&mg, g_out, batch, H, W) ||
      !halo_map(&mh, h_out ? h_out : g_out, batch, H, W)) {
    fprintf(stderr, "tat_conv_mid_bwd_weights: tensor map encoding failed\n");
    return TAT_ERR_CUDA;
  }
  int ctas_used = ctas;
  if (h_out) {
    if (!smem_attr<k_conv_mid_wgrad<true>>(wgrad_smem_bytes())) return TAT_ERR_CUDA;
    tat::pdl_launch(true, k_conv_mid_wgrad<true>, ctas, 288, wgrad_smem_bytes(), s, batch, H, W, mi, mg, mh, scratch);
  } else {  // an already masked gradient: tcgen05, one CTA per SM
    CUtensorMap tg, ti;
    if (!wgrad_tc_map(&tg, g_out, batch, H, W, wg::GX, wg::GY) ||
        !wgrad_tc_map(&ti, h_in, batch, H, W, wg::IX, wg::IY)) {
      fprintf(stderr, "tat_conv_mid_bwd_weights: tensor map encoding failed\n");
      return TAT_ERR_CUDA;
    }
    const long long tiles = (long long)batch * ((H + wg::TY - 1) / wg::TY) * ((W + wg::TX - 1) / wg::TX + 1);
    ctas_used = (int)(tiles < wg::CTAS ? tiles : wg::CTAS);
    if (!smem_attr<k_conv_mid_wgrad_tc>(wg::SMEM)) return TAT_ERR_CUDA;
    tat::pdl_launch(true, k_conv_mid_wgrad_tc, ctas_used, 192, wg::SMEM, s, batch, H, W, tg, ti, scratch);
  }
  tat_status st = launched("tat_conv_mid_bwd_weights");
  if (st != TAT_OK) return st;
  tat::pdl_launch(true, k_reduce_partials, (nw + 31) / 32, 1024, 0, s, ctas_used, 9 * C * C, C, scratch, gw, gb);
  return launched("tat_conv_mid_bwd_weights");
}

tat_status tat_conv_out_fwd(int batch, int H, int W, const tat_bf16* h, const tat_bf16* w, const float* b,
                            const float* residual, float* out, tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || !h || !w || !b || !residual || !out || misaligned(h)) return TAT_ERR_INVALID_ARG;
  CUtensorMap mh;
  if (!halo_map(&mh, h, batch, H, W)) {
    fprintf(stderr, "tat_conv_out_fwd: tensor map encoding failed\n");
    return TAT_ERR_CUDA;
  }
  if (!smem_attr<k_conv_out_fwd>(out_fwd_smem_bytes())) return TAT_ERR_CUDA;
  tat::pdl_launch(true, k_conv_out_fwd, thin_ctas(batch, H, W, 3), 256, out_fwd_smem_bytes(), static_cast<cudaStream_t>(stream), batch, H, W, mh, w, b, residual, out);
  return launched("tat_conv_out_fwd");
}

tat_status tat_conv_out_bwd(int batch, int H, int W, const float* g_out, const tat_bf16* h, const tat_bf16* w,
                            int mask_relu, tat_bf16* g_h, float* scratch, size_t scratch_floats, float* gw, float* gb,
                            tat_stream_t stream) {
  if (bad_sizes(batch, H, W) || !g_out || !h || !w || !g_h || !scratch || !gw || !gb || misaligned(h))
    return TAT_ERR_INVALID_ARG;
  const int ctas = thin_ctas(batch, H, W, 2);
  if (scratch_floats < (size_t)ctas * (9 * C + 1)) return TAT_ERR_INVALID_ARG;
  CUtensorMap mh;
  if (!halo_map(&mh, h, batch, H, W)) {
    fprintf(stderr, "tat_conv_out_bwd: tensor map encoding failed\n");
    return TAT_ERR_CUDA;
  }
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (mask_relu) {
    if (!smem_attr<k_conv_out_bwd<true>>(out_bwd_smem_bytes())) return TAT_ERR_CUDA;
    tat::pdl_launch(true, k_conv_out_bwd<true>, ctas, 256, out_bwd_smem_bytes(), s, batch, H, W, mh, g_out, w, g_h, scratch);
  } else {
    if (!smem_attr<k_conv_out_bwd<false>>(out_bwd_smem_bytes())) return TAT_ERR_CUDA;
    tat::pdl_launch(true, k_conv_out_bwd<false>, ctas, 256, out_bwd_smem_bytes(), s, batch, H, W, mh, g_out, w, g_h, scratch);
  }
  tat_status st = launched("tat_conv_out_bwd");
  if (st != TAT_OK) return st;
  tat::pdl_launch(true, k_reduce_partials, (9 * C + 1 + 31) / 32, 1024, 0, s, ctas, 9 * C, 1, scratch, gw, gb);
  return launched("tat_conv_out_bwd");
}

tat_status tat_adam(long long count, float lr, float beta1, float beta2, float eps, int step, float* param,
                    const float* grad, float* m, float* v, tat_bf16* w_bf16, tat_stream_t stream) {
  if (count <= 0 || step < 1 || !param || !grad || !m || !v) return TAT_ERR_INVALID_ARG;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  tat::pdl_launch(true, k_adam, blocks_for(count, 256), 256, 0, static_cast<cudaStream_t>(stream), count, lr, beta1, beta2, eps, c1, c2, param, grad, m, v, w_bf16);
  return launched("tat_adam");
}

tat_status tat_fill(long long count, float value, float* out, tat_stream_t stream) {
  if (count <= 0 || !out) return TAT_ERR_INVALID_ARG;
  tat::pdl_launch(true, k_fill, blocks_for(count, 256), 256, 0, static_cast<cudaStream_t>(stream), count, value, out);
  return launched("tat_fill");
}

tat_status tat_to_bf16(long long count, const float* x, tat_bf16* out, tat_stream_t stream) {
  if (count <= 0 || !x || !out) return TAT_ERR_INVALID_ARG;
  tat::pdl_launch(true, k_to_bf16, blocks_for(count, 256), 256, 0, static_cast<cudaStream_t>(stream), count, x, out);
  return launched("tat_to_bf16");
}

tat_status tat_mse(long long count, const float* a, const float* b, float scale, float* grad, float* loss,
                   tat_stream_t stream) {
  if (count <= 0 || !a || !b || !loss) return TAT_ERR_INVALID_ARG;
  tat::pdl_launch(true, k_mse, blocks_for(count, 256), 256, 0, static_cast<cudaStream_t>(stream), count, a, b, scale, grad, loss);
  return launched("tat_mse");
}

}  // extern "C"
