/*
 * tat_lpd.h -- kernels of the learned primal-dual reconstruction (Section
 * 4.2.1, Eqs. LPD_dual, LPD_primal, emp_loss): the 3x3 convolution layers of
 * the dual net Gamma (on the data grid n_det x n_t) and the primal net Lambda
 * (on the image grid n x n), their backward passes, the loss and the optimizer
 * step.  The operators inside the unrolled iterations are tat_forward_batched
 * and tat_adjoint_batched.
 *
 * Each net is three 3x3 convolutions with zero padding (stride 1, same size):
 *   in  layer: cin FP32 planes (cin = 3 for Gamma: q, A f, y; 2 for Lambda: f, A* q)
 *              -> 32 channels, bias, ReLU
 *   mid layer: 32 -> 32 channels, bias, ReLU
 *   out layer: 32 -> 1 channel, bias, added to the residual (q or f):
 *              q_{k+1} = q_k + Gamma(q_k, A f_k, y),  f_{k+1} = f_k + Lambda(f_k, A* q_{k+1}).
 * Convolution means cross-correlation: out(y, x) = sum over dy, dx in {-1,0,1}
 * of w[tap] * in(y+dy, x+dx), tap = 3 (dy+1) + (dx+1).
 *
 * Precision: BF16 operands (inputs rounded to BF16 as they are read, weights
 * stored in BF16, hidden activations and their gradients stored in BF16),
 * FP32 accumulation, FP32 biases, residual planes, outputs of the out layer,
 * gradients of the FP32 planes and of all weights.  All layers run on the
 * tensor cores (BF16 x BF16 -> FP32, exact products): the 32 -> 32 forward and
 * the data gradient of an already masked gradient on tcgen05 (accumulators in
 * tensor memory), the others on mma.sync m16n8k16; the FP32 gradient entering
 * the out layer's backward is split into two BF16 terms (hi + lo, 16
 * significand bits).  Tiles of the hidden activations are staged by TMA, so
 * those pointers (h, h_in, h_out, g_h, g_out of the BF16 layers), and the
 * weights w of the 32 -> 32 layer (read in 16-byte words), must be 16-byte
 * aligned (TAT_ERR_INVALID_ARG otherwise).
 *
 * Layouts (all DEVICE pointers owned by the caller): planes FP32 [batch][H][W];
 * hidden activations BF16 NHWC [batch][H][W][32] (BF16 as its 16-bit pattern,
 * unsigned short); weights: in [9][cin][32], mid [9][32 out][32 in], out
 * [9][32]; biases FP32 [32], [32], [1].  Gradient outputs for weights and
 * biases are ACCUMULATED (+=), so one buffer collects the gradients of the
 * weight-shared blocks of all unrolled iterations.  Kernels that reduce over
 * pixels write per-CTA partial sums into `scratch` (FP32, at least
 * tat_lpd_scratch_floats(batch, H, W) floats) and then add them in a fixed
 * order: the sums are deterministic.  Calls are asynchronous on `stream`;
 * TAT_ERR_INVALID_ARG for NULL required pointers, non-positive sizes, grids of
 * batch x H x W >= 2^31 pixels, cin not 2 or 3, or a scratch buffer that is too
 * small.
 */
#ifndef TAT_LPD_H_
#define TAT_LPD_H_

#include <stddef.h>

#include "tat.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef unsigned short tat_bf16; /* bit pattern of a bfloat16 value */

/* Floats of scratch the weight-gradient kernels need for this problem size. */
size_t tat_lpd_scratch_floats(int batch, int H, int W);

/* h = relu(conv_in(x0, x1[, x2]) + b).  x2 is NULL when cin == 2. */
tat_status tat_conv_in_fwd(int batch, int H, int W, int cin, const float* x0, const float* x1, const float* x2,
                           const tat_bf16* w, const float* b, tat_bf16* h, tat_stream_t stream);
/* gx_c (+)= d/dx_c of <g_h, h> through the ReLU (mask h > 0); gx_c may be NULL;
 * bit c of `accumulate` set adds into gx_c, clear overwrites it.  h == NULL here
 * and below: g_h is already masked (tat_conv_mid_bwd_data with h_in writes it so). */
tat_status tat_conv_in_bwd_data(int batch, int H, int W, int cin, const tat_bf16* g_h, const tat_bf16* h,
                                const tat_bf16* w, float* gx0, float* gx1, float* gx2, int accumulate,
                                tat_stream_t stream);
tat_status tat_conv_in_bwd_weights(int batch, int H, int W, int cin, const float* x0, const float* x1,
                                   const float* x2, const tat_bf16* g_h, const tat_bf16* h, float* scratch,
                                   size_t scratch_floats, float* gw, float* gb, tat_stream_t stream);
/* Both of the above in one pass over g_h and h: the data-plane gradients (skipped when
 * gx0, gx1 and gx2 are all NULL; w may then be NULL) and the weight gradients (skipped when
 * gw is NULL; x0, x1, x2 (cin == 3), scratch and gb are then required). */
tat_status tat_conv_in_bwd(int batch, int H, int W, int cin, const float* x0, const float* x1, const float* x2,
                           const tat_bf16* g_h, const tat_bf16* h, const tat_bf16* w, float* gx0, float* gx1,
                           float* gx2, int accumulate, float* scratch, size_t scratch_floats, float* gw, float* gb,
                           tat_stream_t stream);

/* h_out = relu(conv_mid(h_in) + b)  (tensor cores). */
tat_status tat_conv_mid_fwd(int batch, int H, int W, const tat_bf16* h_in, const tat_bf16* w, const float* b,
                            tat_bf16* h_out, tat_stream_t stream);
/* g_in = d/dh_in of <g_out, h_out> through the ReLU (tensor cores; BF16 output).
 * h_out == NULL: g_out is already the gradient of the pre-activation (masked by
 * the ReLU, as tat_conv_out_bwd with mask_relu writes it).  h_in != NULL: g_in
 * is multiplied by [h_in > 0], i.e. it is the gradient of the in layer's
 * pre-activation (h_in being that layer's ReLU output). */
tat_status tat_conv_mid_bwd_data(int batch, int H, int W, const tat_bf16* g_out, const tat_bf16* h_out,
                                 const tat_bf16* w, const tat_bf16* h_in, tat_bf16* g_in, tat_stream_t stream);
/* gw += d/dw, gb += d/db of <g_out, h_out> (tensor cores; h_out == NULL as above: then
 * on tcgen05, one CTA per SM, with the taps of a kernel row and four pixel shifts stacked
 * into one MMA; with h_out, on mma.sync). */
tat_status tat_conv_mid_bwd_weights(int batch, int H, int W, const tat_bf16* h_in, const tat_bf16* g_out,
                                    const tat_bf16* h_out, float* scratch, size_t scratch_floats, float* gw,
                                    float* gb, tat_stream_t stream);

/* out = residual + conv_out(h) + b; out may alias residual. */
tat_status tat_conv_out_fwd(int batch, int H, int W, const tat_bf16* h, const tat_bf16* w, const float* b,
                            const float* residual, float* out, tat_stream_t stream);
/* g_h = d/dh <g_out, out> (BF16), times [h > 0] when mask_relu != 0 (then g_h is
 * the gradient of the mid layer's pre-activation, h being that layer's ReLU
 * output); gw += d/dw, gb += d/db.  (d/d residual = g_out.) */
tat_status tat_conv_out_bwd(int batch, int H, int W, const float* g_out, const tat_bf16* h, const tat_bf16* w,
                            int mask_relu, tat_bf16* g_h, float* scratch, size_t scratch_floats, float* gw, float* gb,
                            tat_stream_t stream);

/* TAT_ERR_TIMEOUT (and the flag cleared) if a tensor-core convolution gave up
 * waiting for one of its TMA tile copies since the last call, else TAT_OK.
 * Synchronises with the device. */
tat_status tat_lpd_check(void);

/* Test of the give-up path: one thread waits, at most `tries` (1 .. 2^20) times, on an
 * mbarrier that nothing arrives on, then sets the flag tat_lpd_check reports and writes 1 to
 * *gave_up (a DEVICE int).  The context stays usable.  Asynchronous on `stream`. */
tat_status tat_lpd_timeout_probe(int tries, int* gave_up, tat_stream_t stream);

/* Adam step (bias-corrected, step >= 1) on FP32 parameters; w_bf16 (optional)
 * receives the updated parameters rounded to BF16. */
tat_status tat_adam(long long count, float lr, float beta1, float beta2, float eps, int step, float* param,
                    const float* grad, float* m, float* v, tat_bf16* w_bf16, tat_stream_t stream);

/* out[i] = value for i < count. */
tat_status tat_fill(long long count, float value, float* out, tat_stream_t stream);

/* Copies FP32 values to BF16 (round to nearest even). */
tat_status tat_to_bf16(long long count, const float* x, tat_bf16* out, tat_stream_t stream);

/* *loss += scale * sum (a - b)^2 (device scalar); grad (optional) = 2 scale (a - b)
 * (Eq. emp_loss with scale = 1 / (number of pixels)). */
tat_status tat_mse(long long count, const float* a, const float* b, float scale, float* grad, float* loss,
                   tat_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* TAT_LPD_H_ */
