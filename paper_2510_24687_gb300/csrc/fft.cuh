// Shared-memory FFT core for the stages of Algorithms 1 and 2.
//
// Stockham autosort, decimation in time, mixed radix 8/4/3/2, natural order in
// and out, unnormalised.  Each pass reads R elements with stride L/R, applies
// the twiddles e^{-+2 pi i r (j mod Ns)/(Ns R)} from an FP64-derived table,
// does a radix-R DFT in registers, synchronises, and writes the results back
// in place at (j - j mod Ns) R + j mod Ns + r Ns.  A group of `nthr` threads
// works on one transform; every thread holds at most 16 values per pass.
// The buffer index is padded by one element per 32 to spread the strided
// accesses over the shared-memory banks.
#pragma once

#include <cuda_runtime.h>

#include "plan.hpp"

namespace tat {

__device__ __forceinline__ int spad(int i) { return i + (i >> 5); }
__host__ __device__ __forceinline__ int spad_len(int L) { return L + (L >> 5) + 1; }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int R, bool INV>
__device__ __forceinline__ void bfly(float2* v);

template <>
__device__ __forceinline__ void bfly<2, false>(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <>
__device__ __forceinline__ void bfly<2, true>(float2* v) {
  bfly<2, false>(v);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = mul_mi<INV>(csub(x1, x3));
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, d);
  x3 = csub(b, d);
}
template <>
__device__ __forceinline__ void bfly<4, false>(float2* v) { dft4<false>(v[0], v[1], v[2], v[3]); }
template <>
__device__ __forceinline__ void bfly<4, true>(float2* v) { dft4<true>(v[0], v[1], v[2], v[3]); }

template <bool INV>
__device__ __forceinline__ void dft8(float2* v) {
  const float s2 = 0.70710678118654752440f;
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // o_k *= e^{-+ 2 pi i k/8}
  o1 = INV ? make_float2(s2 * (o1.x - o1.y), s2 * (o1.x + o1.y)) : make_float2(s2 * (o1.x + o1.y), s2 * (o1.y - o1.x));
  o2 = mul_mi<INV>(o2);
  o3 = INV ? make_float2(-s2 * (o3.x + o3.y), s2 * (o3.x - o3.y)) : make_float2(s2 * (o3.y - o3.x), -s2 * (o3.x + o3.y));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}
template <>
__device__ __forceinline__ void bfly<8, false>(float2* v) { dft8<false>(v); }
template <>
__device__ __forceinline__ void bfly<8, true>(float2* v) { dft8<true>(v); }

template <bool INV>
__device__ __forceinline__ void dft3(float2* v) {
  const float s3 = 0.86602540378443864676f;
  float2 a = v[0], b = v[1], c = v[2];
  float2 s = cadd(b, c);
  float2 t = make_float2(a.x - 0.5f * s.x, a.y - 0.5f * s.y);
  float2 d = csub(b, c);
  // -i*s3*d (forward) or +i*s3*d (inverse)
  float2 u = INV ? make_float2(-s3 * d.y, s3 * d.x) : make_float2(s3 * d.y, -s3 * d.x);
  v[0] = cadd(a, s);
  v[1] = cadd(t, u);
  v[2] = csub(t, u);
}
template <>
__device__ __forceinline__ void bfly<3, false>(float2* v) { dft3<false>(v); }
template <>
__device__ __forceinline__ void bfly<3, true>(float2* v) { dft3<true>(v); }

template <int R, bool INV>
__device__ __forceinline__ void fft_pass(float2* buf, int L, int Ns, const float2* __restrict__ tw, int tid,
                                         int nthr) {
  constexpr int NB = 16 / R;
  const int nb = L / R;
  const int tws = L / (Ns * R);
  const bool act = tid < nthr;
  float2 v[NB][R];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tid + b * nthr;
    if (act && j < nb) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = buf[spad(j + r * nb)];
      if (Ns > 1) {
        const int k = j % Ns;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = __ldg(&tw[k * r * tws]);
          v[b][r] = INV ? cmulc(v[b][r], w) : cmul(v[b][r], w);
        }
      }
      bfly<R, INV>(v[b]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tid + b * nthr;
    if (act && j < nb) {
      const int k = j % Ns;
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[spad(base + r * Ns)] = v[b][r];
    }
  }
  __syncthreads();
}

// Radix schedule of a length L = 2^k 3^m: all radix-3 passes, then radix-8
// passes, then radix-4 passes (a trailing 8*2 is done as 4*4), then at most
// one radix-2 pass.  The plan builder uses the same rule.
template <int L>
struct Sched {
  static constexpr int pow3(int x) { return x % 3 == 0 ? 1 + pow3(x / 3) : 0; }
  static constexpr int strip3(int x) { return x % 3 == 0 ? strip3(x / 3) : x; }
  static constexpr int log2i(int x) { return x <= 1 ? 0 : 1 + log2i(x / 2); }
  static constexpr int n3 = pow3(L);
  static constexpr int k = log2i(strip3(L));
  static constexpr int n8 = (k % 3 == 1 && k >= 4) ? k / 3 - 1 : k / 3;
  static constexpr int n4 = (k % 3 == 1) ? (k >= 4 ? 2 : 0) : (k % 3 == 2 ? 1 : 0);
  static constexpr int n2 = (k % 3 == 1 && k < 4) ? 1 : 0;
};

// Compile-time length: every pass is unrolled with constant strides.
template <int L, bool INV>
__device__ __forceinline__ void fft_ct(float2* buf, const float2* __restrict__ tw, int tid, int nthr) {
  using S = Sched<L>;
  int Ns = 1;
#pragma unroll
  for (int s = 0; s < S::n3; ++s) { fft_pass<3, INV>(buf, L, Ns, tw, tid, nthr); Ns *= 3; }
#pragma unroll
  for (int s = 0; s < S::n8; ++s) { fft_pass<8, INV>(buf, L, Ns, tw, tid, nthr); Ns *= 8; }
#pragma unroll
  for (int s = 0; s < S::n4; ++s) { fft_pass<4, INV>(buf, L, Ns, tw, tid, nthr); Ns *= 4; }
  if (S::n2) fft_pass<2, INV>(buf, L, Ns, tw, tid, nthr);
}

// Runtime length (any 2^k 3^m): the same schedule read from the plan.
template <bool INV>
__device__ __forceinline__ void fft_run(float2* buf, const FftDev& f, int tid, int nthr) {
  const int L = f.L;
  int Ns = 1, s = 0;
#pragma unroll 1
  for (; s < f.npass && f.radix[s] == 3; ++s, Ns *= 3) fft_pass<3, INV>(buf, L, Ns, f.tw, tid, nthr);
#pragma unroll 1
  for (; s < f.npass && f.radix[s] == 8; ++s, Ns *= 8) fft_pass<8, INV>(buf, L, Ns, f.tw, tid, nthr);
#pragma unroll 1
  for (; s < f.npass && f.radix[s] == 4; ++s, Ns *= 4) fft_pass<4, INV>(buf, L, Ns, f.tw, tid, nthr);
  if (s < f.npass && f.radix[s] == 2) fft_pass<2, INV>(buf, L, Ns, f.tw, tid, nthr);
}

// L > 0: compile-time schedule (must equal f.L); L == 0: runtime schedule.
template <int L, bool INV>
__device__ __forceinline__ void fft(float2* buf, const FftDev& f, int tid, int nthr) {
  if constexpr (L == 0) fft_run<INV>(buf, f, tid, nthr);
  else fft_ct<L, INV>(buf, f.tw, tid, nthr);
}

}  // namespace tat
