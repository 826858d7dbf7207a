// Shared-memory FFT core for the stages of Algorithms 1 and 2.
//
// Stockham autosort, decimation in time, mixed radix 16/8/4/3/2, natural order
// in and out, unnormalised.  Each pass reads R elements with stride L/R,
// applies the twiddles e^{-+2 pi i r (j mod Ns)/(Ns R)}, does a radix-R DFT in
// registers, synchronises, and writes the results back in place at
// (j - j mod Ns) R + j mod Ns + r Ns.  A group of `nthr` threads works on one
// transform; every thread holds at most 16 values per pass.
//
// * Twiddles: one to four exact values per butterfly come from an FP64-derived
//   table (w^1, w^2, w^4, w^8); the other powers are products of at most three
//   of them.
// * The buffer index is padded by one element per 16, which makes the strided
//   stores of radix-16 passes free of shared-memory bank conflicts.
// * Pruning: the first pass reads only indices < n_in (the rest is taken as
//   zero and never touched), the last pass writes only indices < n_out.
// * `pre` multiplies the input by conj(pre[i]) in the first pass and `post`
//   multiplies the output by post[o] in the last pass (either may be null).
#pragma once

#include <cuda_runtime.h>

#include "plan.hpp"

namespace tat {

__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }
// spad(i + r s) = spad(i) + r spad(s) for i >= 0 when s is a multiple of 16: the padded
// slots of a butterfly's strided elements then sit at a constant step (immediate offsets).
__device__ __forceinline__ bool spad_linear(int s) { return (s & 15) == 0; }
__host__ __device__ __forceinline__ int spad_len(int L) { return L + (L >> 4) + 1; }

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

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = mul_mi<INV>(csub(x1, x3));
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, d);
  x3 = csub(b, d);
}

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

// a * e^{-+ 2 pi i E/16} for the exponents a 16-point DFT needs.
template <int E, bool INV>
__device__ __forceinline__ float2 w16(float2 a) {
  constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, s2 = 0.70710678118654752440f;
  constexpr float cr = E == 1 ? c1 : E == 2 ? s2 : E == 3 ? s1 : E == 6 ? -s2 : E == 9 ? -c1 : 1.f;
  constexpr float si = E == 1 ? -s1 : E == 2 ? -s2 : E == 3 ? -c1 : E == 6 ? -s2 : E == 9 ? s1 : 0.f;
  const float wi = INV ? -si : si;
  return make_float2(a.x * cr - a.y * wi, a.x * wi + a.y * cr);
}

template <bool INV>
__device__ __forceinline__ void dft16(float2* v) {
  // x[n1 + 4 n2]: DFT4 over n2 for each n1, twiddle w16^(n1 k2), DFT4 over n1.
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) dft4<INV>(v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]);
  // v[n1 + 4 k2] now holds y[n1][k2]
  v[5] = w16<1, INV>(v[5]);
  v[6] = w16<2, INV>(v[6]);
  v[7] = w16<3, INV>(v[7]);
  v[9] = w16<2, INV>(v[9]);
  v[10] = mul_mi<INV>(v[10]);
  v[11] = w16<6, INV>(v[11]);
  v[13] = w16<3, INV>(v[13]);
  v[14] = w16<6, INV>(v[14]);
  v[15] = w16<9, INV>(v[15]);
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) dft4<INV>(v[4 * k2], v[4 * k2 + 1], v[4 * k2 + 2], v[4 * k2 + 3]);
  // v[4 k2 + k1] holds X[4 k1 + k2]; transpose the 4 x 4 block in registers
  float2 t;
  t = v[1]; v[1] = v[4]; v[4] = t;
  t = v[2]; v[2] = v[8]; v[8] = t;
  t = v[3]; v[3] = v[12]; v[12] = t;
  t = v[6]; v[6] = v[9]; v[9] = t;
  t = v[7]; v[7] = v[13]; v[13] = t;
  t = v[11]; v[11] = v[14]; v[14] = t;
}

// cos(2 pi j / 32), j = 0..31 (sin(2 pi j / 32) = entry (j + 24) mod 32).
__device__ constexpr float kCos32[32] = {
    1.f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
    0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f, 0.19509032201612826785f,
    0.f, -0.19509032201612826785f, -0.38268343236508977173f, -0.55557023301960222474f,
    -0.70710678118654752440f, -0.83146961230254523708f, -0.92387953251128675613f, -0.98078528040323044913f,
    -1.f, -0.98078528040323044913f, -0.92387953251128675613f, -0.83146961230254523708f,
    -0.70710678118654752440f, -0.55557023301960222474f, -0.38268343236508977173f, -0.19509032201612826785f,
    0.f, 0.19509032201612826785f, 0.38268343236508977173f, 0.55557023301960222474f,
    0.70710678118654752440f, 0.83146961230254523708f, 0.92387953251128675613f, 0.98078528040323044913f};

// 32-point DFT: two 16-point DFTs of the even and odd samples and one radix-2 step
// X[k] = E[k] + w^k O[k], X[k + 16] = E[k] - w^k O[k], w = e^{-+2 pi i / 32}.
template <bool INV>
__device__ __forceinline__ void dft32(float2* v) {
  float2 e[16], o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft16<INV>(e);
  dft16<INV>(o);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float c = kCos32[k], sn = kCos32[(k + 24) & 31];
    const float2 w = make_float2(c, INV ? sn : -sn);
    const float2 t = cmul(o[k], w);
    v[k] = cadd(e[k], t);
    v[k + 16] = csub(e[k], t);
  }
}

template <int R, bool INV>
__device__ __forceinline__ void bfly(float2* v) {
  if constexpr (R == 32) {
    dft32<INV>(v);
  } else if constexpr (R == 16) {
    dft16<INV>(v);
  } else if constexpr (R == 8) {
    dft8<INV>(v);
  } else if constexpr (R == 4) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  } else if constexpr (R == 3) {
    const float s3 = 0.86602540378443864676f;
    float2 a = v[0], b = v[1], c = v[2];
    float2 s = cadd(b, c);
    float2 t = make_float2(a.x - 0.5f * s.x, a.y - 0.5f * s.y);
    float2 d = csub(b, c);
    float2 u = INV ? make_float2(-s3 * d.y, s3 * d.x) : make_float2(s3 * d.y, -s3 * d.x);
    v[0] = cadd(a, s);
    v[1] = cadd(t, u);
    v[2] = csub(t, u);
  } else {
    dft2<INV>(v[0], v[1]);
  }
}

// Multiplies v[r] by w^r (INV: conj(w)^r), r = 1..R-1, for the butterfly
// twiddle w = tw[base].  w^1, w^2, w^4, w^8 are read from the table; every other
// power is a product of at most three of them, formed just before it is used
// so that few twiddles are live at once.
template <int R, bool INV>
__device__ __forceinline__ void apply_twiddles(float2* v, const float2* __restrict__ tw, int base) {
  auto mul = [](float2 a, float2 w) { return INV ? cmulc(a, w) : cmul(a, w); };
  const float2 w1 = __ldg(&tw[base]);
  v[1] = mul(v[1], w1);
  if constexpr (R >= 3) {
    const float2 w2 = __ldg(&tw[2 * base]);
    v[2] = mul(v[2], w2);
    if constexpr (R >= 4) {
      const float2 w3 = cmul(w1, w2);
      v[3] = mul(v[3], w3);
      if constexpr (R >= 8) {
        const float2 w4 = __ldg(&tw[4 * base]);
        v[4] = mul(v[4], w4);
        v[5] = mul(v[5], cmul(w4, w1));
        v[6] = mul(v[6], cmul(w4, w2));
        v[7] = mul(v[7], cmul(w4, w3));
        if constexpr (R >= 16) {
          const float2 w8 = __ldg(&tw[8 * base]);
          v[8] = mul(v[8], w8);
          v[9] = mul(v[9], cmul(w8, w1));
          v[10] = mul(v[10], cmul(w8, w2));
          v[11] = mul(v[11], cmul(w8, w3));
          const float2 w12 = cmul(w8, w4);
          v[12] = mul(v[12], w12);
          v[13] = mul(v[13], cmul(w12, w1));
          v[14] = mul(v[14], cmul(w12, w2));
          v[15] = mul(v[15], cmul(w12, w3));
        }
      }
    }
  }
}

// Same as apply_twiddles, with w^1, w^2, w^4, w^8 supplied by the caller.
template <int R, bool INV>
__device__ __forceinline__ void apply_twiddles_given(float2* v, float2 w1, float2 w2, float2 w4, float2 w8) {
  auto mul = [](float2 a, float2 w) { return INV ? cmulc(a, w) : cmul(a, w); };
  v[1] = mul(v[1], w1);
  if constexpr (R >= 3) v[2] = mul(v[2], w2);
  if constexpr (R >= 4) {
    const float2 w3 = cmul(w1, w2);
    v[3] = mul(v[3], w3);
    if constexpr (R >= 8) {
      v[4] = mul(v[4], w4);
      v[5] = mul(v[5], cmul(w4, w1));
      v[6] = mul(v[6], cmul(w4, w2));
      v[7] = mul(v[7], cmul(w4, w3));
      if constexpr (R >= 16) {
        v[8] = mul(v[8], w8);
        v[9] = mul(v[9], cmul(w8, w1));
        v[10] = mul(v[10], cmul(w8, w2));
        v[11] = mul(v[11], cmul(w8, w3));
        const float2 w12 = cmul(w8, w4);
        v[12] = mul(v[12], w12);
        v[13] = mul(v[13], cmul(w12, w1));
        v[14] = mul(v[14], cmul(w12, w2));
        v[15] = mul(v[15], cmul(w12, w3));
      }
    }
  }
}

// Base powers w^1, w^2, w^4, w^8 of twiddle index k < Ns from a per-pass
// shared-memory table (layout in FftDev); only the powers radix R needs.
template <int R>
__device__ __forceinline__ void pass_tw(const float2* t, int Ns, int k, float2& w1, float2& w2, float2& w4,
                                        float2& w8) {
  if (Ns <= 16 || (Ns & 15)) {
    w1 = t[k];
    if constexpr (R >= 3) w2 = t[Ns + k];
    if constexpr (R >= 8) w4 = t[2 * Ns + k];
    if constexpr (R >= 16) w8 = t[3 * Ns + k];
  } else {
    const int na = Ns >> 4, a = k >> 4, b = k & 15;
    const float2* lo = t + 4 * na;
    w1 = cmul(t[a], lo[b]);
    if constexpr (R >= 3) w2 = cmul(t[na + a], lo[16 + b]);
    if constexpr (R >= 8) w4 = cmul(t[2 * na + a], lo[32 + b]);
    if constexpr (R >= 16) w8 = cmul(t[3 * na + a], lo[48 + b]);
  }
}

// keep_mod > 0: the next pass is the last, with Ns = keep_mod, and keeps only its outputs
// below n_out, which read exactly the values at o with o mod keep_mod < n_out: the others
// are not written.
template <int R, bool INV>
__device__ __forceinline__ void fft_pass(float2* buf, int L, int Ns, const float2* __restrict__ tw, int tid,
                                         int nthr, bool first, bool last, int n_in, int n_out,
                                         const float2* __restrict__ pre, const float2* __restrict__ post,
                                         const float2* ptws = nullptr, int keep_mod = 0) {
  constexpr int NB = 16 / R;
  const int nb = L / R;
  const int tws = L / (Ns * R);
  const bool act = tid < nthr;
  float2 v[NB][R];
  const bool lin_in = spad_linear(nb), lin_out = spad_linear(Ns);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tid + b * nthr;
    if (act && j < nb) {
      const int sj = spad(j);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int idx = j + r * nb;
        const int slot = lin_in ? sj + r * spad(nb) : spad(idx);
        if (first) {
          float2 x = idx < n_in ? buf[slot] : make_float2(0.f, 0.f);
          if (pre != nullptr && idx < n_in) x = cmulc(x, __ldg(&pre[idx]));
          v[b][r] = x;
        } else {
          v[b][r] = buf[slot];
        }
      }
      if (Ns > 1) {
        if (ptws != nullptr) {
          float2 w1 = make_float2(1.f, 0.f), w2 = w1, w4 = w1, w8 = w1;
          pass_tw<R>(ptws, Ns, j % Ns, w1, w2, w4, w8);
          apply_twiddles_given<R, INV>(v[b], w1, w2, w4, w8);
        } else {
          apply_twiddles<R, INV>(v[b], tw, (j % Ns) * tws);
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
      const int sb = spad(base);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int o = base + r * Ns;
        const int slot = lin_out ? sb + r * spad(Ns) : spad(o);
        if (last) {
          if (o < n_out) buf[slot] = post != nullptr ? cmul(v[b][r], __ldg(&post[o])) : v[b][r];
        } else if (keep_mod > 0) {
          if (o % keep_mod < n_out) buf[slot] = v[b][r];
        } else {
          buf[slot] = v[b][r];
        }
      }
    }
  }
  __syncthreads();
}

// Radix schedule of a length L = 2^k 3^m: all radix-3 passes, then radix-16
// passes, then the remainder of k mod 4 as 8*4 (one 16 fewer), 4 or 8, or a
// single 2 for k = 1 (order V = 0); order V = 1 runs the same passes in reverse
// (the tail radix first, the radix-3 passes last).  The plan builder uses the
// same rule (fft_schedule), and the autotuner picks the order per plan.
template <int L, int V = 0>
struct Sched {
  __host__ __device__ static constexpr int pow3(int x) { return x % 3 == 0 ? 1 + pow3(x / 3) : 0; }
  __host__ __device__ static constexpr int strip3(int x) { return x % 3 == 0 ? strip3(x / 3) : x; }
  __host__ __device__ static constexpr int log2i(int x) { return x <= 1 ? 0 : 1 + log2i(x / 2); }
  static constexpr int n3 = pow3(L);
  static constexpr int k = log2i(strip3(L));
  static constexpr int n16full = k / 4, rem = k % 4;
  static constexpr int n16 = (rem == 1 && n16full >= 1) ? n16full - 1 : n16full;
  static constexpr int ntail = rem == 0 ? 0 : (rem == 1 && n16full >= 1) ? 2 : 1;
  static constexpr int npass = n3 + n16 + ntail;
  __host__ __device__ static constexpr int radix0(int s) {
    return s < n3 ? 3
         : s < n3 + n16 ? 16
         : rem == 1 ? (n16full >= 1 ? (s == n3 + n16 ? 8 : 4) : 2)
         : rem == 2 ? 4
         : 8;
  }
  __host__ __device__ static constexpr int radix(int s) { return V == 0 ? radix0(s) : radix0(npass - 1 - s); }
};

template <int L, bool INV, int S, int NS, int V = 0>
__device__ __forceinline__ void fft_ct_from(float2* buf, const FftDev& f, int tid, int nthr, int n_in, int n_out,
                                            const float2* pre, const float2* post, const float2* smptw) {
  if constexpr (S < Sched<L, V>::npass) {
    constexpr int R = Sched<L, V>::radix(S);
    fft_pass<R, INV>(buf, L, NS, f.tw, tid, nthr, S == 0, S == Sched<L, V>::npass - 1, n_in, n_out, pre, post,
                     smptw != nullptr && S > 0 ? smptw + f.ptw_off[S] : nullptr);
    fft_ct_from<L, INV, S + 1, NS * R, V>(buf, f, tid, nthr, n_in, n_out, pre, post, smptw);
  }
}

// Runtime length (any 2^k 3^m): the same schedule read from the plan.
template <bool INV>
__device__ __forceinline__ void fft_run(float2* buf, const FftDev& f, int tid, int nthr, int n_in, int n_out,
                                        const float2* pre, const float2* post, const float2* smptw) {
  const int L = f.L;
  int Ns = 1;
#pragma unroll 1
  for (int s = 0; s < f.npass; ++s) {
    const int R = f.radix[s];
    const bool first = s == 0, last = s == f.npass - 1;
    const float2* pt = smptw != nullptr && s > 0 ? smptw + f.ptw_off[s] : nullptr;
    switch (R) {
      case 16: fft_pass<16, INV>(buf, L, Ns, f.tw, tid, nthr, first, last, n_in, n_out, pre, post, pt); break;
      case 8: fft_pass<8, INV>(buf, L, Ns, f.tw, tid, nthr, first, last, n_in, n_out, pre, post, pt); break;
      case 4: fft_pass<4, INV>(buf, L, Ns, f.tw, tid, nthr, first, last, n_in, n_out, pre, post, pt); break;
      case 3: fft_pass<3, INV>(buf, L, Ns, f.tw, tid, nthr, first, last, n_in, n_out, pre, post, pt); break;
      default: fft_pass<2, INV>(buf, L, Ns, f.tw, tid, nthr, first, last, n_in, n_out, pre, post, pt); break;
    }
    Ns *= R;
  }
}

// L > 0: compile-time schedule of order V (must equal f's schedule); L == 0: runtime
// schedule read from f.  Reads buf[0, n_in), writes buf[0, n_out); every thread of the
// CTA must call it.  `smptw`: shared-memory copy of f.ptw (null: global twiddle table).
template <int L, bool INV, int V = 0>
__device__ __forceinline__ void fft(float2* buf, const FftDev& f, int tid, int nthr, int n_in, int n_out,
                                    const float2* pre = nullptr, const float2* post = nullptr,
                                    const float2* smptw = nullptr) {
  if constexpr (L == 0) fft_run<INV>(buf, f, tid, nthr, n_in, n_out, pre, post, smptw);
  else fft_ct_from<L, INV, 0, 1, V>(buf, f, tid, nthr, n_in, n_out, pre, post, smptw);
}

// First pass of a compile-time schedule with its inputs from `load(i)` (global memory,
// or zero where the caller knows an input vanishes) instead of the shared buffer:
// the copy into shared memory and the first pass's reads become one step.  Ns = 1, so
// no twiddles; the outputs go to the buffer at j R + r.
template <int R, bool INV, class Load>
__device__ __forceinline__ void fft_pass_load(float2* buf, int L, int tid, int nthr, Load& load) {
  constexpr int NB = 16 / R;
  const int nb = L / R;
  const bool act = tid < nthr;
  float2 v[NB][R];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tid + b * nthr;
    if (act && j < nb) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = load(j + r * nb);
      bfly<R, INV>(v[b]);
    }
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tid + b * nthr;
    if (act && j < nb) {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[spad(j * R + r)] = v[b][r];
    }
  }
  __syncthreads();
}

// Last pass (Ns R = L) handing each output o < n_out to `store(o, value)` instead of
// writing it back to the buffer, which it leaves unchanged (no trailing barrier).  The
// outputs of butterfly j are j + r L/R, so butterflies j >= n_out are skipped whole
// (with the radix-3 pass last and n_out = L/6, half of them).
template <int R, bool INV, class Store>
__device__ __forceinline__ void fft_pass_store(const float2* buf, int L, int tid, int nthr, int n_out, Store& store,
                                               const float2* ptws) {
  constexpr int NB = 16 / R;
  const int nb = L / R;  // = Ns
  const bool act = tid < nthr;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const int j = tid + b * nthr;
    if (act && j < nb && j < n_out) {
      float2 v[R];
      const int sj = spad(j);
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = buf[spad_linear(nb) ? sj + r * spad(nb) : spad(j + r * nb)];
      float2 w1 = make_float2(1.f, 0.f), w2 = w1, w4 = w1, w8 = w1;
      pass_tw<R>(ptws, nb, j, w1, w2, w4, w8);
      apply_twiddles_given<R, INV>(v, w1, w2, w4, w8);
      bfly<R, INV>(v);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (j + r * nb < n_out) store(j + r * nb, v[r]);
    }
  }
}

template <int L, bool INV, int V, int S, int NS, class Load, class Store>
__device__ __forceinline__ void fft_io_from(float2* buf, const FftDev& f, int tid, int nthr, int n_out, Load& load,
                                            Store& store, const float2* smptw) {
  constexpr int NP = Sched<L, V>::npass;
  if constexpr (S < NP) {
    constexpr int R = Sched<L, V>::radix(S);
    if constexpr (S == 0) {
      fft_pass_load<R, INV>(buf, L, tid, nthr, load);
    } else if constexpr (S == NP - 1) {
      fft_pass_store<R, INV>(buf, L, tid, nthr, n_out, store, smptw + f.ptw_off[S]);
    } else {
      // the pass before the last writes only what the kept outputs of the last one read
      constexpr int keep = S == NP - 2 ? L / Sched<L, V>::radix(NP - 1) : 0;
      fft_pass<R, INV>(buf, L, NS, f.tw, tid, nthr, false, false, 0, keep > 0 ? n_out : 0, nullptr, nullptr,
                       smptw + f.ptw_off[S], keep < n_out ? 0 : keep);
    }
    fft_io_from<L, INV, V, S + 1, NS * R>(buf, f, tid, nthr, n_out, load, store, smptw);
  }
}

// Unnormalised DFT of length L (compile-time schedule of at least two passes) from
// load(i), i < L, to store(o, X[o]) for o < n_out, with `buf` (xpad_len(L) slots) as
// the exchange between passes and `smptw` the shared-memory per-pass twiddles (loaded
// and synchronised by the caller).  Every thread of the CTA must call it.
template <int L, bool INV, int V = 0, class Load, class Store>
__device__ __forceinline__ void fft_io(float2* buf, const FftDev& f, int tid, int nthr, int n_out, Load load,
                                       Store store, const float2* smptw) {
  static_assert(L > 0 && Sched<L, V>::npass >= 2, "fft_io needs a compile-time schedule of two or more passes");
  fft_io_from<L, INV, V, 0, 1>(buf, f, tid, nthr, n_out, load, store, smptw);
}

// Copies an FFT's per-pass twiddle tables to shared memory (caller syncs).
__device__ __forceinline__ void load_pass_tw(float2* dst, const FftDev& f, int tid, int nthr) {
  for (int i = tid; i < f.ptw_len; i += nthr) dst[i] = f.ptw[i];
}

}  // namespace tat

namespace tat {

// ------------------------------------------------------------------------
// In-place four-step DFT of length N = RA * 256 (RA in {2, 4, 8, 16}) for the
// column transforms, where a column's spectrum stays in shared memory.
//   n = 256 n1 + n2, k = k1 + RA k2, k2 = k21 + 16 k22:
//   step A : per n2, DFT_RA over n1, twiddle w_N^(n2 k1)          (256 threads)
//   step B1: per (k1, m2), DFT16 over m1 of y[k1][16 m1 + m2],
//            twiddle w_256^(m2 k21)                                (16 threads/block)
//   step B2: per (k1, k21), DFT16 over m2                          (same warp)
// Every thread reads and writes back the same set of positions in each step,
// so only two CTA barriers are needed.  The output stays in the permuted
// layout colpos(q) = 256 k1 + 16 k21 + k22, which the resampling reads and
// writes directly.  The inverse runs the conjugate transposes in reverse.
template <int L>
struct FourStep {
  static constexpr bool on = L == 512 || L == 1024 || L == 2048 || L == 4096 || L == 8192;
  static constexpr int RA = on ? L / 256 : 1;
};
// Steps A and B are looped when a group has fewer threads than 256 (step A)
// or RA*16 (step B); group sizes are multiples of 32, so every lane of a warp
// runs the same iterations of step B and __syncwarp stays warp-uniform.

// Shared-memory slot of element i of a transform buffer of length L: one pad
// slot per 16 elements (the Stockham passes), and for the four-step lengths one
// more per 256, so that the permuted layout's neighbouring bins q, q+1 (256
// slots apart) fall into different banks when a warp walks q.
template <int L>
__device__ __forceinline__ int xpad(int i) {
  if constexpr (FourStep<L>::on) return i + (i >> 4) + (i >> 8);
  else return i + (i >> 4);
}
__host__ __device__ __forceinline__ int xpad_len(int L) {
  const bool four = L == 512 || L == 1024 || L == 2048 || L == 4096 || L == 8192;
  return L + (L >> 4) + (four ? (L >> 8) : 0) + 1;
}

// Position of FFT bin q of a column buffer (identity for other lengths).
template <int L>
__device__ __forceinline__ int colpos(int q) {
  if constexpr (FourStep<L>::on) {
    constexpr int RA = FourStep<L>::RA;
    const int k1 = q & (RA - 1), r = q / RA;
    return 256 * k1 + 16 * (r & 15) + (r >> 4);
  } else {
    return q;
  }
}

// Twiddle tables of the four-step transform, 192 float2 per transform length
// (FP64-computed in the plan; copied to shared memory once per CTA):
//   [  0, 64): w_N^(16 a p), a < 16, p in {1,2,4,8}   (step A, high digit of n2)
//   [ 64,128): w_N^(b p),    b < 16                   (step A, low digit of n2)
//   [128,192): w_256^(m p),  m < 16                   (step B1)
// stored as [p][a], [p][b], [p][m] with p index 0..3 for powers 1, 2, 4, 8.
constexpr int kFourStepTw = 192;

__device__ __forceinline__ void load_fourstep_tw(float2* smtw, const float2* __restrict__ g, int tid, int nthr) {
  for (int i = tid; i < kFourStepTw; i += nthr) smtw[i] = g[i];
}

__device__ __forceinline__ void stepA_tw(const float2* smtw, int n2, float2& w1, float2& w2, float2& w4, float2& w8) {
  const int a = n2 >> 4, b = n2 & 15;
  w1 = cmul(smtw[a], smtw[64 + b]);
  w2 = cmul(smtw[16 + a], smtw[80 + b]);
  w4 = cmul(smtw[32 + a], smtw[96 + b]);
  w8 = cmul(smtw[48 + a], smtw[112 + b]);
}

// e^{-+2 pi i k / R} (R in {2, 4, 8, 16, 32}; INV takes the + sign) from the 32nd roots of unity.
template <int R, bool INV>
__device__ __forceinline__ float2 unit_root(int k) {
  const int j = (k * (32 / R)) & 31;
  const float s = kCos32[(j + 24) & 31];  // sin(2 pi j / 32) = cos(2 pi (j - 8) / 32)
  return make_float2(kCos32[j], INV ? s : -s);
}

// Step A twiddles v[k1] *= w^(k1 n2) (INV: conjugate) from w^(n2 p), p = 1, 2, 4, 8; for
// RA = 32 the power 16 is the square of the power 8.
template <int RA, bool INV>
__device__ __forceinline__ void stepA_apply(float2* v, float2 w1, float2 w2, float2 w4, float2 w8) {
  if constexpr (RA <= 16) {
    apply_twiddles_given<RA, INV>(v, w1, w2, w4, w8);
  } else {
    static_assert(RA == 32, "four-step lengths are RA * 256 with RA <= 32");
    apply_twiddles_given<16, INV>(v, w1, w2, w4, w8);
    const float2 w16 = cmul(w8, w8);
#pragma unroll
    for (int r = 16; r < 32; ++r) v[r] = INV ? cmulc(v[r], w16) : cmul(v[r], w16);
    apply_twiddles_given<16, INV>(v + 16, w1, w2, w4, w8);
  }
}

// Forward: x[0, n_in) in natural order -> X[q] * post[q] at colpos(q).
// When n_in <= 512 only the inputs n1 = 0, 1 of the DFT_RA of step A are
// non-zero (the zero padding of the rows and columns), and step A reduces to
// X[k1] = x0 + x1 e^{-2 pi i k1 / RA}; the inverse likewise keeps only the
// outputs n1 = 0, 1 when n_out <= 512.
// `smtw`: the shared-memory copy of the four-step twiddle table; `nthr`: the
// threads of the calling group (tid < nthr, all take part in the four-step
// loops); `sthr` (<= nthr): the thread count of the Stockham fallback.
template <int L>
__device__ __forceinline__ void col_fft_fwd(float2* buf, const FftDev& f, const float2* smtw, int tid, int nthr,
                                            int sthr, int n_in, const float2* __restrict__ post) {
  if constexpr (!FourStep<L>::on) {
    fft<L, false>(buf, f, tid, sthr, n_in, f.L, nullptr, post);
  } else {
    constexpr int RA = FourStep<L>::RA;
    for (int n2 = tid; n2 < 256; n2 += nthr) {
      float2 v[RA];
      if (n_in <= 512) {
        const float2 x0 = n2 < n_in ? buf[xpad<L>(n2)] : make_float2(0.f, 0.f);
        const float2 x1 = 256 + n2 < n_in ? buf[xpad<L>(256 + n2)] : make_float2(0.f, 0.f);
#pragma unroll
        for (int k1 = 0; k1 < RA; ++k1) v[k1] = cadd(x0, cmul(x1, unit_root<RA, false>(k1)));
      } else {
#pragma unroll
        for (int n1 = 0; n1 < RA; ++n1) {
          const int idx = 256 * n1 + n2;
          v[n1] = idx < n_in ? buf[xpad<L>(idx)] : make_float2(0.f, 0.f);
        }
        bfly<RA, false>(v);
      }
      float2 w1, w2, w4, w8;
      stepA_tw(smtw, n2, w1, w2, w4, w8);
      stepA_apply<RA, false>(v, w1, w2, w4, w8);
#pragma unroll
      for (int k1 = 0; k1 < RA; ++k1) buf[xpad<L>(256 * k1 + n2)] = v[k1];
    }
    __syncthreads();
    for (int t = tid; t < RA * 16; t += nthr) {
      const int blk = t >> 4, m = t & 15;
      const int base = 256 * blk;
      float2 v[16];
#pragma unroll
      for (int m1 = 0; m1 < 16; ++m1) v[m1] = buf[xpad<L>(base + 16 * m1 + m)];
      bfly<16, false>(v);
      apply_twiddles_given<16, false>(v, smtw[128 + m], smtw[144 + m], smtw[160 + m], smtw[176 + m]);
#pragma unroll
      for (int k21 = 0; k21 < 16; ++k21) buf[xpad<L>(base + 16 * k21 + m)] = v[k21];
      __syncwarp();
#pragma unroll
      for (int m2 = 0; m2 < 16; ++m2) v[m2] = buf[xpad<L>(base + 16 * m + m2)];
      bfly<16, false>(v);
#pragma unroll
      for (int k22 = 0; k22 < 16; ++k22) {
        float2 x = v[k22];
        if (post != nullptr) x = cmul(x, __ldg(&post[blk + RA * (m + 16 * k22)]));
        buf[xpad<L>(base + 16 * m + k22)] = x;
      }
    }
    __syncthreads();
  }
}

struct NoMid {
  __device__ __forceinline__ void operator()() const {}
};
// The barrier among the threads that run a transform: the whole CTA by default; a named
// barrier of one warp group in a warp-specialised kernel.
struct CtaBar {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// Inverse (unnormalised): Z[q] at colpos(q), times conj(pre[q]) -> z[0, n_out) in natural order.
// `mid()` runs between the two steps of the four-step transform (before the transform for
// other lengths): a place to issue global loads whose latency the second step hides.
template <int L, class Mid = NoMid, class Bar = CtaBar>
__device__ __forceinline__ void col_fft_inv(float2* buf, const FftDev& f, const float2* smtw, int tid, int nthr,
                                            int sthr, int n_out, const float2* __restrict__ pre, Mid mid = Mid{},
                                            Bar bar = Bar{}) {
  if constexpr (!FourStep<L>::on) {
    mid();
    fft<L, true>(buf, f, tid, sthr, f.L, n_out, pre, nullptr);
  } else {
    constexpr int RA = FourStep<L>::RA;
    for (int t = tid; t < RA * 16; t += nthr) {
      const int blk = t >> 4, m = t & 15;
      const int base = 256 * blk;
      float2 v[16];
#pragma unroll
      for (int k22 = 0; k22 < 16; ++k22) {
        float2 x = buf[xpad<L>(base + 16 * m + k22)];
        if (pre != nullptr) x = cmulc(x, __ldg(&pre[blk + RA * (m + 16 * k22)]));
        v[k22] = x;
      }
      bfly<16, true>(v);
#pragma unroll
      for (int m2 = 0; m2 < 16; ++m2) buf[xpad<L>(base + 16 * m + m2)] = v[m2];
      __syncwarp();
#pragma unroll
      for (int k21 = 0; k21 < 16; ++k21) v[k21] = buf[xpad<L>(base + 16 * k21 + m)];
      apply_twiddles_given<16, true>(v, smtw[128 + m], smtw[144 + m], smtw[160 + m], smtw[176 + m]);
      bfly<16, true>(v);
#pragma unroll
      for (int m1 = 0; m1 < 16; ++m1) buf[xpad<L>(base + 16 * m1 + m)] = v[m1];
    }
    bar();
    mid();
    for (int n2 = tid; n2 < 256; n2 += nthr) {
      float2 v[RA];
#pragma unroll
      for (int k1 = 0; k1 < RA; ++k1) v[k1] = buf[xpad<L>(256 * k1 + n2)];
      float2 w1, w2, w4, w8;
      stepA_tw(smtw, n2, w1, w2, w4, w8);
      stepA_apply<RA, true>(v, w1, w2, w4, w8);
      if (n_out <= 512) {
        float2 o0 = v[0], o1 = v[0];
#pragma unroll
        for (int k1 = 1; k1 < RA; ++k1) {
          o0 = cadd(o0, v[k1]);
          o1 = cadd(o1, cmul(v[k1], unit_root<RA, true>(k1)));
        }
        if (n2 < n_out) buf[xpad<L>(n2)] = o0;
        if (256 + n2 < n_out) buf[xpad<L>(256 + n2)] = o1;
      } else {
        bfly<RA, true>(v);
#pragma unroll
        for (int n1 = 0; n1 < RA; ++n1)
          if (256 * n1 + n2 < n_out) buf[xpad<L>(256 * n1 + n2)] = v[n1];
      }
    }
    bar();
  }
}

}  // namespace tat
