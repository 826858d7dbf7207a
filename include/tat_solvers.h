/*
 * tat_solvers.h -- fused element-wise steps of the variational solvers that
 * call A and A* every iteration (Section 4.2), and their backward passes for
 * differentiating through unrolled iterations.
 *
 * Problem (Eq. minim with R = TV, f >= 0, and the fidelity halved as in the
 * dual step Eq. PDHG-dual):
 *     min_{f >= 0, f = Pi_Omega0 f}  1/2 ||A f - g||^2 + alpha ||grad f||_1
 *
 * NNLS (alpha = 0) is projected gradient descent (Eqs. NNLS, NNLS-projstep,
 * projectionHalfCircle):
 *     f <- Pi_Omega0 max(0, f - lambda A*(A f - g)).
 *
 * TV-LS is the primal-dual hybrid gradient method of Chambolle and Pock
 * (Eqs. PDHG-dual, PDHG-primal, PDHG-relaxation).  Reading: the paper
 * applies prox of alpha*TV inside the primal update without naming an inner
 * solver; here the TV term goes to the dual side, K = [A; s grad_h], so no
 * inner iterations are needed (s > 0 is a free balancing scale; the TV bound
 * becomes alpha/s):
 *     q     <- (q + sigma (A fbar - g)) / (1 + sigma)
 *     p     <- proj_{|p| <= alpha/s} (p + sigma s grad_h fbar)      (pointwise)
 *     f_new <- Pi_Omega0 max(0, f - tau (A* q - s div_h p))
 *     fbar  <- 2 f_new - f                                      (theta = 1)
 * grad_h: forward differences divided by h, zero across the last column (x)
 * and last row (y); div_h = -grad_h^T.  In the calls below the caller passes
 * h_eff = h / s, so that "grad_h" and "div_h" there include s.
 *
 * Arrays are DEVICE float arrays owned by the caller.  Images are n x n,
 * row-major (f[iy*n + ix]), `batch` images at stride n*n.  Dual gradient
 * fields hold two n x n planes per image, x then y, at stride 2*n*n.  `mask`
 * (an n x n array of 0/1 shared by the batch, Pi_Omega0) may be NULL.
 * Output arrays may alias the input of the same role (in-place update) but
 * no other argument.  Calls are asynchronous on `stream`.  Errors:
 * TAT_ERR_INVALID_ARG for a NULL required pointer or a non-positive size,
 * step or bound; TAT_ERR_CUDA if a launch fails.
 */
#ifndef TAT_SOLVERS_H_
#define TAT_SOLVERS_H_

#include <stddef.h>

#include "tat.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Projected gradient step (Eq. NNLS-projstep; with Eq. projectionHalfCircle
 * when mask != NULL): out[i] = mask[i % mask_period] * max(lo, a*x[i] + b*y[i])
 * for i < count.  y may be NULL (taken as 0); lo = -INFINITY disables the
 * clamp.  With a = 1, b = -1, lo = -INFINITY it forms the residual A f - g. */
tat_status tat_axpby_clamp(long long count, float a, const float* x, float b, const float* y, float lo,
                           const float* mask, long long mask_period, float* out, tat_stream_t stream);

/* Backward of tat_axpby_clamp, given its output `out`:
 *   G = mask * [out > lo] * grad_out;  grad_x = a*G;  grad_y = b*G.
 * grad_x or grad_y may be NULL (not wanted).  At a kink (out == lo) the
 * zero subgradient is taken. */
tat_status tat_axpby_clamp_backward(long long count, const float* out, float lo, const float* mask,
                                    long long mask_period, const float* grad_out, float a, float* grad_x, float b,
                                    float* grad_y, tat_stream_t stream);

/* Data dual step (Eq. PDHG-dual): q_out = (q_in + sigma (Af - g)) / (1 + sigma).
 * Linear; its backward is three tat_axpby_clamp scalings. */
tat_status tat_pd_dual_data(long long count, float sigma, const float* Af, const float* g, const float* q_in,
                            float* q_out, tat_stream_t stream);

/* TV dual step: p_out = proj_{|p| <= bound}(p_in + sigma grad_h fbar), with
 * h = h_eff and |.| the pointwise Euclidean norm of the (x, y) pair. */
tat_status tat_tv_dual(int batch, int n, float h_eff, float sigma, float bound, const float* fbar, const float* p_in,
                       float* p_out, tat_stream_t stream);

/* Backward of tat_tv_dual: with u = p_in + sigma grad_h fbar and P the
 * projection, grad_p_in = DP(u)^T grad_p_out and grad_fbar = sigma grad_h^T
 * grad_p_in = -sigma div_h grad_p_in.  DP(u) = I if |u| <= bound, else
 * (bound/|u|)(I - u u^T/|u|^2).  grad_fbar may be NULL. */
tat_status tat_tv_dual_backward(int batch, int n, float h_eff, float sigma, float bound, const float* fbar,
                                const float* p_in, const float* grad_p_out, float* grad_p_in, float* grad_fbar,
                                tat_stream_t stream);

/* Primal step (Eqs. PDHG-primal and PDHG-relaxation, theta = 1):
 *   f_out = mask * max(0, f_in - tau (Asq - div_h p));  fbar = 2 f_out - f_in,
 * with Asq = A* q and h = h_eff.  f_out may alias f_in. */
tat_status tat_tv_primal(int batch, int n, float h_eff, float tau, const float* Asq, const float* p,
                         const float* mask, const float* f_in, float* f_out, float* fbar, tat_stream_t stream);

/* Backward of tat_tv_primal, given its output f_out:
 *   D = mask * [f_out > 0] * (grad_f_out + 2 grad_fbar)
 *   grad_f_in = D - grad_fbar;  grad_Asq = -tau D;  grad_p = -tau grad_h D.
 * grad_f_out or grad_fbar may be NULL (taken as 0). */
tat_status tat_tv_primal_backward(int batch, int n, float h_eff, float tau, const float* f_out, const float* mask,
                                  const float* grad_f_out, const float* grad_fbar, float* grad_f_in, float* grad_Asq,
                                  float* grad_p, tat_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TAT_SOLVERS_H_ */
