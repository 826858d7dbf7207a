/*
 * tat_debug.h -- host-only introspection of the FP64 plan tables of libtat.
 *
 * These calls run on the CPU and touch no GPU.  They expose the FP64 values
 * from which the device tables are rounded, so that tests can compare them
 * with independent evaluations.  None of them is needed to apply A or A*.
 */
#ifndef TAT_DEBUG_H_
#define TAT_DEBUG_H_

#include "tat.h"

#ifdef __cplusplus
extern "C" {
#endif

/* J_k(x) for k = 0..kmax (out has kmax+1 doubles), as the plan evaluates the
 * Bessel table that Section 3.1 precomputes: the DFT of the samples of the
 * Jacobi-Anger expansion (Eq. Anger), e^{i x sin tau} = sum_k J_k(x) e^{ik tau}. */
tat_status tat_debug_bessel(double x, int kmax, double* out);

/* Nodes (in units of the radial step dlam) and weights of the quadrature the
 * plan uses for the angular modes k = -1, 0, 1 (Section 3.1: a rule whose
 * discretisation points cluster toward lambda = 0; the paper does not give
 * it).  *count receives the number of nodes; the arrays are written only when
 * both are non-NULL and *count is at least that number on entry. */
tat_status tat_debug_low_mode_rule(double* nodes, double* weights, int* count);

/* Bilinear stencil (Section 3.1, Algorithm 1 step 3) of `count` half-plane
 * polar samples: ring r (1..J radial nodes, J+1.. low-mode nodes) and
 * half-circle index lp (phi = 2 pi (lp - n_phi/4)/n_phi).  Writes the stencil
 * column i0 and row k0 (signed frequency indices) and the weights a, b in
 * [0, 1), in FP64 exactly as the plan computes them before rounding. */
tat_status tat_debug_stencils(const tat_plan_desc* desc, int* ring, int* lp, int* i0, int* k0, double* a,
                              double* b, int count);

/* Same work as tat_forward_batched / tat_adjoint_batched, and additionally
 * records events[0] on `stream` before the first stage and events[s] after
 * stage s, s = 1..5 (forward: rows, columns, rings, modes, detectors; adjoint:
 * detectors, modes, rings, columns, rows).  `events` holds 6 caller-created
 * cudaEvent_t handles; the calls are for per-stage timing only. */
tat_status tat_debug_forward_batched_timed(tat_plan_t plan, int batch, const float* f, long long f_stride,
                                           float* g, long long g_stride, void* workspace, tat_stream_t stream,
                                           void* const* events);
tat_status tat_debug_adjoint_batched_timed(tat_plan_t plan, int batch, const float* g, long long g_stride,
                                           float* f, long long f_stride, void* workspace, tat_stream_t stream,
                                           void* const* events);
/* tat_inverse_batched with 7 events: before the first stage and after each of
 * detectors, modes (sine transform), rings, columns, rows, and the constant C. */
tat_status tat_debug_inverse_batched_timed(tat_plan_t plan, int batch, const float* g, long long g_stride,
                                           float* f, long long f_stride, void* workspace, tat_stream_t stream,
                                           void* const* events);

#ifdef __cplusplus
}
#endif
#endif /* TAT_DEBUG_H_ */
