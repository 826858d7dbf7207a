/*
 * tat.h -- C ABI of the fast circular-geometry PAT/TAT operators A and A*.
 *
 * Method: Hauptmann, Kunyansky, Poimala, "Fast algorithms enabling
 * optimization and deep learning for photoacoustic tomography in a circular
 * detection geometry" (arXiv 2510.24687).
 *
 *   A  : f -> g,  the trace on the detector circle of the solution of the
 *        wave equation with initial pressure f and zero initial velocity
 *        (Section 1, Eqs. wave-eq / Cauchy; Section 2.1, Eq. green_conv),
 *        computed by Algorithm 1 in O(n^2 log n) flops.
 *   A* : g -> f,  the adjoint of A for the inner products of
 *        Eq. innerProducts (Section 2.1, Eq. adjoint), computed with the
 *        stages of Algorithm 2 as the exact transpose of the discrete A.
 *
 * Units and grids (all entry points):
 *   image  f[iy*n + ix] at (x, y) = (-R + ix*2R/(n-1), -R + iy*2R/(n-1)),
 *          ix, iy = 0..n-1 (node-centred n x n grid covering [-R, R]^2);
 *          values outside the support disk |x| <= support_radius*R are
 *          ignored by A and returned as 0 by A*.
 *   data   g[d*n_t + m] = g(t_m, z_d) with t_m = m*T/(n_t-1), m = 0..n_t-1,
 *          and z_d = R(cos th_d, sin th_d), th_d = 2*pi*d/n_det (detector-major);
 *          detectors outside the arc Gamma read and write 0.
 *   A* is the adjoint for <u,v>_X = int u v dx and <h,k>_Y = int int h k dz dt,
 *          discretised with weights h^2 per pixel and dt * 2*pi*R/n_det per
 *          sample, so that <A f, g>_Y = <f, A* g>_X holds for the discrete maps.
 *
 * Memory and ownership: every f, g and workspace pointer is a DEVICE pointer
 * on the device that was current when the plan was created; the caller owns
 * them.  The plan owns its device tables (immutable after creation, so one
 * plan may be used concurrently from several streams, each call with its own
 * workspace).  Calls are asynchronous on the given stream (a cudaStream_t
 * passed as void*; NULL means the legacy default stream).
 *
 * Errors: every call returns a tat_status; nothing is thrown across the ABI.
 * Launch errors are returned as TAT_ERR_CUDA; asynchronous faults surface at
 * the next synchronising call.  Precision: device arithmetic is FP32; every
 * table (per-mode Bessel kernel, interpolation stencils and weights, twiddles,
 * phases, low-mode quadrature) is computed in FP64 on the host and rounded.
 */
#ifndef TAT_H_
#define TAT_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tat_plan_s* tat_plan_t;  /* opaque */
typedef void* tat_stream_t;             /* a cudaStream_t */

typedef enum {
  TAT_OK = 0,
  TAT_ERR_INVALID_ARG = 1, /* bad size, non-positive c/R/T, NULL pointer, bad stride */
  TAT_ERR_UNSUPPORTED = 2, /* valid arguments outside what this build implements     */
  TAT_ERR_OOM = 3,         /* device or host allocation failed                       */
  TAT_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed            */
  TAT_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up                     */
  TAT_ERR_INTERNAL = 6     /* an internal consistency check failed                   */
} tat_status;

/* Problem statement (Section 2.1) plus the discretisation parameters of
 * Section 3.1.  tat_plan_desc_default fills the paper's defaults. */
typedef struct {
  int n;                  /* image is n x n, n >= 8                                        */
  int n_det;              /* detectors equispaced on the full circle, even, >= 8            */
  int n_t;                /* time samples on [0, T], >= 8                                   */
  double c;               /* speed of sound, > 0                                            */
  double R;               /* detector-circle radius, > 0                                    */
  double T;               /* observation window (0, T], > 0                                 */
  double support_radius;  /* Omega_0 = disk of this radius / R (paper: 0.98, Section 4.1)    */
  double arc_begin;       /* Gamma = th in [arc_begin, arc_begin + arc_len), radians        */
  double arc_len;         /* 2*pi (full circle) by default                                  */
  int n_phi;              /* angular samples of the polar grid; 0 -> n_det (paper)          */
  double pad_L;           /* half-width L of the padded square, in units of R; 0 -> T_new+2 */
  int low_mode_quadrature;/* 1: clustered quadrature for k = -1,0,1 (Section 3.1); 0: off   */
} tat_plan_desc;

/* Grid integers chosen by the plan (for tests and tooling). */
typedef struct {
  int N;       /* padded square is N x N nodes (smallest 2^a 3^b >= 2L/h, even)  */
  int M;       /* extended time T_new = M*dt (smallest 2^a 3^b >= max(2T,6)/dt)  */
  int J;       /* radial nodes lambda_j = j*pi/T_new, j = 0..J                    */
  int n_phi;   /* angular nodes of the polar grid                                 */
  int K;       /* angular modes kept, k = -K..K (K = n_phi/2)                      */
  int n_low;   /* extra radial nodes of the low-mode quadrature                   */
  int n_points;/* half-plane polar points resampled per image                     */
  double h, dt, dlam, dxi, lam_c;
} tat_plan_info;

/* Host only (no CUDA call): validates *desc and reports the grid integers a
 * plan would use, following the grid rules of Section 3.1. */
tat_status tat_plan_query(const tat_plan_desc* desc, tat_plan_info* info);

/* Fills *desc with the paper's defaults for the given problem (Section 3.1). */
tat_status tat_plan_desc_default(tat_plan_desc* desc, int n, int n_det, int n_t,
                                 double c, double R, double T);

/* Creates a plan on the current CUDA device: derives the grids, evaluates the
 * Bessel table J_|k|(lambda_j) for k = 0..K once (Section 3.1, end) and every
 * other table in FP64, rounds them to FP32 and uploads them.  On failure
 * *plan is set to NULL. */
tat_status tat_plan_create(tat_plan_t* plan, int n, int n_det, int n_t,
                           double c, double R, double T);
tat_status tat_plan_create_ex(tat_plan_t* plan, const tat_plan_desc* desc);
tat_status tat_plan_destroy(tat_plan_t plan);
tat_status tat_plan_get_info(tat_plan_t plan, tat_plan_info* info);

/* Bytes of device workspace a call with this batch size needs (0 on error).
 * The workspace must be 256-byte aligned; its contents need no initialisation. */
size_t tat_workspace_size(tat_plan_t plan, int batch);

/* g = A f  (Algorithm 1).  f: n*n floats, g: n_det*n_t floats. */
tat_status tat_forward(tat_plan_t plan, const float* f, float* g, void* workspace,
                       tat_stream_t stream);

/* f = A* g  (Algorithm 2, exact transpose of Algorithm 1).  g: n_det*n_t, f: n*n. */
tat_status tat_adjoint(tat_plan_t plan, const float* g, float* f, void* workspace,
                       tat_stream_t stream);

/* Batched variants: image b starts at f + b*f_stride, data b at g + b*g_stride
 * (strides in floats, >= n*n and >= n_det*n_t respectively).  One launch per
 * stage covers the whole batch; the workspace is tat_workspace_size(plan, batch). */
tat_status tat_forward_batched(tat_plan_t plan, int batch, const float* f, long long f_stride,
                               float* g, long long g_stride, void* workspace,
                               tat_stream_t stream);
tat_status tat_adjoint_batched(tat_plan_t plan, int batch, const float* g, long long g_stride,
                               float* f, long long f_stride, void* workspace,
                               tat_stream_t stream);

/* f ~ A^{-1} g  (Algorithm 3): the universal backprojection formula for data
 * on (0, T) x Gamma extended by zero (Eq. approx_UBP), computed on the grids of
 * A*: detector DFT (Eq. FourSerForg), sine transform in t, the per-mode factor
 * -2 (-i)^|k| J'_|k|(lambda) of Eq. Four_coef_v (the paper prints -4 pi; the
 * 2 pi belongs to the transform of G used in its appendix, and -2 is the value
 * consistent with Eq. green_conv: A^{-1} A f = f for full data as T grows),
 * the angular series, bilinear polar -> Cartesian interpolation in
 * (lambda, phi), the 2D inverse DFT, then Pi_Omega0 (v + C) with C the
 * negative mean of v over the disk |x| <= R outside Omega_0 (Eq.
 * silly_integral; C = 0 when that set has no grid node).  The result does not
 * depend on c and R beyond T' = cT/R.  Requires n_phi == n_det (the default),
 * else TAT_ERR_UNSUPPORTED.  g: n_det*n_t floats, f: n*n floats; workspace as
 * for A*.  A left inverse on complete data (Gamma the full circle, T large);
 * on partial data it is the paper's approximate reconstruction. */
tat_status tat_inverse(tat_plan_t plan, const float* g, float* f, void* workspace, tat_stream_t stream);
tat_status tat_inverse_batched(tat_plan_t plan, int batch, const float* g, long long g_stride,
                               float* f, long long f_stride, void* workspace, tat_stream_t stream);

/* g = A f for one image, like tat_forward, but with no workspace argument: the
 * scratch lives in a static 16 MiB device buffer inside the library.  The
 * paper has no counterpart; this exists for callers that cannot allocate
 * device memory when they need A (a process whose GPU memory is all handed to
 * its own pool, or a loop that cannot afford cudaMalloc's implicit device
 * synchronisation).  The call itself allocates nothing.  Every GPU that loads
 * the library holds the 16 MiB until the process exits.  Every call looks up
 * the buffer's device address on the current device (cudaGetSymbolAddress,
 * which allocates nothing); the first lookup on a device may load the
 * library's device code, so make the first call before any stream capture.
 * f and g must be 4-byte aligned (else TAT_ERR_INVALID_ARG, as for
 * tat_forward).  All calls on a device
 * share the one buffer: calls that overlap on the GPU (different streams or
 * host threads) race and must be serialised by the caller.  Plans whose
 * scratch exceeds 16 MiB (tat_workspace_size(plan, 1)) are rejected with
 * TAT_ERR_UNSUPPORTED; n = 512 with 1024 detectors x 1024 samples fits. */
tat_status tat_forward_noalloc(tat_plan_t plan, const float* f, float* g, tat_stream_t stream);

/* Static string for a status code. */
const char* tat_status_string(tat_status status);

#ifdef __cplusplus
}
#endif
#endif /* TAT_H_ */
