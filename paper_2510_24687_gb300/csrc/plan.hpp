// Internal plan layout shared by the host plan builder (plan.cpp), the CUDA
// kernels (kernels.cu) and the C ABI (capi.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "tat.h"

namespace tat {

// Number of trapezoid nodes j = 0..kLowA-1 replaced by the clustered
// low-mode quadrature, and its number of Gauss-Legendre nodes (Section 3.1:
// "discretization points clustering toward lambda = 0" for k = -1, 0, 1).
constexpr int kLowA = 8;
constexpr int kLowM = 20;

constexpr int kMaxPass = 16;

// One FFT length: radix schedule, its twiddle table e^{-2 pi i k/L}, k < L,
// and the per-pass tables of the base powers w^p, p = 1, 2, 4, 8, that the
// kernels stage in shared memory: for a pass with Ns > 1 and twiddle index
// k < Ns, w = e^{-2 pi i k/(Ns R)}; if Ns <= 16 (or not a multiple of 16) the
// table is direct, [p][k]; otherwise k = 16a + b and w^p = hi[p][a] * lo[p][b]
// with hi of Ns/16 and lo of 16 entries per power.
struct FftDev {
  int L;
  int npass;
  int radix[kMaxPass];
  const float2* tw;
  const float2* ptw;        // concatenated per-pass tables
  int ptw_off[kMaxPass];    // offset of pass s (s >= 1)
  int ptw_len;              // total entries
  const float2* fstw;       // four-step twiddles (192 entries) when L = RA*256, RA in {2,4,8,16}
};

// One half-plane polar sample: polar slot p (ring*nh + l'), stencil row k0
// (signed frequency index) and bilinear weights a, b.  Points are sorted by
// stencil column i0 (implicit in the column offsets), then by k0.
struct PolarEntry {
  int p;
  int k0;
  float a;
  float b;
};

// Slots per warp region of a split column buffer (colsplit.cuh): 32 rows of 17.
constexpr int kSplitRegionSlots = 544;

// The same polar sample for the forward column stage on the split transform, with what the
// gather needs precomputed on the host: the buffer slots of its stencil rows k0 and k0 + 1
// in the split layout, and the phase-weighted row weights (FP64-built, rounded once).
struct PolarEntrySplit {
  int p;           // polar slot
  unsigned slots;  // slot of row k0 (low 16 bits) and of row k0 + 1 (high 16 bits)
  float a;         // weight of the second stencil column
  float pad;
  float2 alpha;    // (1 - b) e^{i k0 dxi}
  float2 beta;     // b e^{i (k0 + 1) dxi}
};

// Everything a kernel needs, passed by value.
struct DevPlan {
  int n, n_det, n_t;
  int N, M, J, n_phi, K, nh;       // K = n_phi/2, nh = n_phi/2 (half circle)
  int n_low, n_rings;              // n_rings = J + 1 + n_low
  int ncol;                        // N/2 half-plane columns
  int low_on;
  float h2_2pi;                    // h^2 / (2 pi)
  float adj_scale;                 // (h^2/2pi) * W_Y / W_X
  FftDev fN, fphi, f2M, fdet;
  const float2* phase;             // [N] e^{i q dxi}, q the signed frequency of FFT bin
  const float2* phase2;            // [ph_lo + 64] two-level form: phase[q] = hi[q >> 6] * lo[q & 63],
                                   // negated for q >= N/2 when ph_flip (hi at 0, lo at ph_lo)
  int ph_lo, ph_flip;
  const int2* rowrange;            // [n] support columns [lo, hi) of each image row
  const float* gamma;              // [n_det] 1 on the arc Gamma, else 0
  const PolarEntry* pts;           // [n_points]
  const PolarEntrySplit* pts_split;  // [n_points] the same points for the split forward column stage
                                     // (null where the split transform does not apply)
  const int* coloff;               // [ncol+1] points with i0 = c: [coloff[c], coloff[c+1])
  const int2* runs;                // [n_runs+1] {first point, k0} of each run of equal k0 within a column,
                                   // column by column; run r ends at runs[r+1].x (a sentinel closes the table)
  const int* runoff;               // [ncol+1] runs of column c: [runoff[c], runoff[c+1])
  const int* pinv;                 // [n_rings x nh] index in pts of polar slot p (-1 for ring 0, which
                                   // has no point): A*'s angular stage writes its polar samples in the
                                   // order of pts, so the scatter reads them contiguously
  const float* Bt;                 // [(K+1) x (J+1)] dlam*lam_j*J_k(lam_j)/n_phi
  const float* Btt;                // Bt by ring tile: [tile][k][g], ring 1 + tile*rpc + g, g < rpc
                                   // (rpc = rings_per_cta_for(n_phi)); each tile padded to bt_bs floats
                                   // (a multiple of 4); zero for rings > J and, with the low-mode rule,
                                   // for k <= 1 and rings < kLowA
  const float* Bit;                // Binv in the same tiled layout (no low-mode zeros)
  int bt_bs;                       // floats per tile block
  const float* Bh;                 // [2 x n_low]     w_q*dlam*lam_q*J_k(lam_q)/n_phi
  const float* Lcos;               // [n_low x n_t]   cos(lam_q t_m)
  const float2* cs_half;           // [nh] (cos phi, sin phi) of the half-circle angles
  // inverse A^{-1} (Algorithm 3)
  const float* Binv;               // [(K+1) x (J+1)] J'_k(lam_j) dt / n_det
  const unsigned* inv_jl;          // [N/2][N/2] quadrant node (c, q): ring j (low 16 bits, 0xffff: beyond
                                   // the cut-off) and angle cell L = floor(atan2(q, c) n_phi / 2pi) (high)
  const float2* inv_ab;            // [N/2][N/2] (a, b): fractional ring and angle positions
  const int* inv_qmax;             // [N/2] largest |q| of column c inside the cut-off (-1: none)
  const int2* outrange;            // [n] columns [lo, hi) of each row inside |x| <= R (the disk Omega)
  float inv_scale;                 // dxi^2 / (2 pi)
  float inv_count;                 // nodes of Omega \ Omega0 (0: no constant C)
  int inv_ok;                      // n_phi == n_det (the inverse keeps the data's own modes)
};

// Tile shapes fixed at compile time per FFT length (index arithmetic by
// shifts); the host uses the same functions for the launch shapes.  Rings per CTA
// in the angular stages: 4 at n_phi = 256, 1024, 2048, 8 at the other compile-time
// lengths below 4096, 2 at 4096, 1 for runtime lengths; time samples per CTA in the
// theta stages: 8 at n_det = 1024, 2048, 16 at the other compile-time lengths below
// 4096, 4 at 4096, 2 for runtime lengths (so that a CTA never exceeds 1024 threads).
// The smaller tiles were measured faster there (more CTAs in flight per SM).
__host__ __device__ constexpr bool ct_angular_length(int L) {
  return L == 64 || L == 128 || L == 256 || L == 512 || L == 1024 || L == 2048;
}
__host__ __device__ constexpr int rings_per_cta_for(int L) {
  return (L == 256 || L == 1024 || L == 2048) ? 4 : ct_angular_length(L) ? 8 : L == 4096 ? 2 : 1;
}
__host__ __device__ constexpr int time_tile_for(int L) {
  return (L == 1024 || L == 2048) ? 8 : ct_angular_length(L) ? 16 : L == 4096 ? 4 : 2;
}

// Launch shapes (host-side knobs; chosen per plan).
struct LaunchCfg {
  int rows_pairs;     // row pairs per CTA in the row pass
  int strip;          // owned columns per CTA in the column pass
  int rings_per_cta;  // rings per CTA in the angular pass
  int t_tile;         // time samples per CTA in the theta pass (even)
  int nt_N, nt_phi, nt_2M, nt_det;  // threads per FFT of each length
  int nt_rows;        // threads per row-pair transform (256 by default for the four-step lengths; 64 or 128
                      // keep more of them busy in the second pass at N <= 1024)
  int cols_threads;   // threads per CTA of the column pass (>= nt_N; fewer than 256 only for four-step lengths)
  int pdl;            // 1: stages launched with programmatic dependent launch (outside graph capture)
  int order_2M;       // pass order of the length-2M FFT of the cosine/sine stages (Sched V: 0 or 1)
  int cols_split;     // bit 0 (A) / bit 1 (A*): that column stage splits each column
                      // transform of length N = 512 RB over the RB warps of a CTA (colsplit.cuh;
                      // RB = 1 .. 16, n <= 512, or 1024 at RB = 16); a clear bit: the four-step one
};

}  // namespace tat

struct tat_plan_s {
  tat_plan_desc desc;
  int device;
  tat::DevPlan d;
  tat::LaunchCfg cfg;
  tat_plan_info info;
  // sizes of the per-image workspace regions, in float2 elements
  size_t ws_x;  // row spectra / per-mode coefficients
  size_t ws_y;  // polar samples / time modes
  tat::FftDev f2M_v[2];  // the length-2M FFT in pass orders 0 and 1; d.f2M is f2M_v[cfg.order_2M]
  int nt_2M_v[2];
  std::vector<void*> allocations;  // device memory owned by the plan
};

namespace tat {
// Grid integers and spacings derived from a plan descriptor (host only).
struct Grids {
  double Tn, h, dt, T_ext, dlam, dxi, lam_c;
  long long M, N, J;
  int n_phi;
  bool low_on;
};
// plan.cpp
tat_status derive_grids(const tat_plan_desc& desc, Grids* g);
void fill_info(const Grids& g, tat_plan_info* info);
tat_status build_plan(const tat_plan_desc& desc, tat_plan_s* plan);
void free_plan(tat_plan_s* plan);
// host-side FP64 helpers (exported for the C ABI self-tests)
void cos_sin_2pi(long long num, long long den, double* c, double* s);
long long smooth_ceil(double x, bool even);
void bessel_orders(double x, int kmax, double* out);
void low_mode_rule(double* nodes, double* weights);
// kernels.cu
tat_status configure_kernels();
tat_status validate_shapes(const tat_plan_s* P);
// `ev` (optional): 6 events recorded before the first and after every stage.
tat_status launch_forward(const tat_plan_s* P, int batch, const float* f, long long fs,
                          float* g, long long gs, void* ws, cudaStream_t st, cudaEvent_t const* ev = nullptr);
tat_status launch_adjoint(const tat_plan_s* P, int batch, const float* g, long long gs,
                          float* f, long long fs, void* ws, cudaStream_t st, cudaEvent_t const* ev = nullptr);
// `ev` (optional): 7 events recorded before the first and after every stage.
tat_status launch_inverse(const tat_plan_s* P, int batch, const float* g, long long gs,
                          float* f, long long fs, void* ws, cudaStream_t st, cudaEvent_t const* ev = nullptr);
}  // namespace tat
