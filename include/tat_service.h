/*
 * tat_service.h -- runtime around the operators of tat.h for many problems of
 * mixed sizes (serving, and solvers that call A / A* / A^{-1} on a stream of
 * requests).  The paper gives the cost structure that makes batching pay
 * (Section 3.3: every stage is a set of independent 1-D transforms per image,
 * O(n^2 log n) per image, plans precomputed once per geometry); the service
 * adds:
 *
 *  - a plan cache per problem descriptor (the Bessel table and stencils are
 *    built once per geometry, as Section 3.1 recommends);
 *  - batching: pending requests with the same descriptor and operation are
 *    launched together, up to max_batch images per launch;
 *  - admission by device memory: every (problem, operation) pair owns a
 *    staging slot (inputs, outputs, workspace) carved from one device arena
 *    of memory_budget bytes; when a slot does not fit, idle slots are evicted
 *    (least recently used first) and then the batch cap of the new slot is
 *    halved until it fits; a request that fits at no batch size completes
 *    with TAT_ERR_OOM;
 *  - one CUDA stream per (problem, operation) pair, so different sizes run
 *    concurrently, and one CUDA graph per (problem, operation, batch) replayed
 *    for every later launch of that shape;
 *  - an autotuner for the launch shapes that the kernels take at run time.
 *
 * Pointers passed to tat_service_submit are owned by the caller: device
 * pointers, or page-locked host pointers (cudaHostAlloc / cudaHostRegister;
 * the staging copies run with cudaMemcpyDefault), in which case a request's
 * upload, operator and download all run on its slot's stream.  They must stay
 * valid, and the output must not be read, until the request has completed
 * (tat_service_synchronize).  Inputs are copied into the
 * slot on the slot's stream after tat_service_flush, so the caller must not
 * modify them before then either.  A service is used from one host thread;
 * completion times are recorded from CUDA host callbacks.
 */
#ifndef TAT_SERVICE_H_
#define TAT_SERVICE_H_

#include <stddef.h>

#include "tat.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tat_service_s* tat_service_t;

/* TAT_OP_PAIR: out = A*(A in), image to image (the gradient of 1/2 |A f - g|^2 at g = 0,
 * the unit of work of the iterative solvers); A in stays in the slot. */
typedef enum { TAT_OP_FORWARD = 0, TAT_OP_ADJOINT = 1, TAT_OP_INVERSE = 2, TAT_OP_PAIR = 3 } tat_op;

typedef struct {
  size_t memory_budget; /* bytes of device memory for all staging slots (one arena) */
  int max_batch;        /* images per launch and per (problem, operation) pair, >= 1 */
  int use_graphs;       /* 1: capture and replay one CUDA graph per (problem, operation, batch) */
  int autotune;         /* 1: run tat_plan_autotune on each new plan at its slot's batch size */
  int one_graph;        /* 1 (with use_graphs): a flush over several sizes or operations whose
                           composition (sizes, operations and batch counts) has been flushed
                           before runs the first batch of each in one CUDA graph, as parallel
                           branches, launched once (captured on the composition's second flush
                           and cached); other flushes, and all with 0, use one graph per
                           (problem, operation, batch) on the slot's own stream */
} tat_service_config;

typedef struct {
  long long requests;   /* submitted */
  long long completed;  /* completed (including failed) */
  long long launches;   /* batched operator launches */
  long long graph_launches;
  long long flush_graphs;   /* single-graph flushes (one_graph): one graph launch for all sizes */
  long long evictions;  /* slots evicted to admit others */
  int plans;            /* plans in the cache */
  int slots;            /* slots resident now */
  size_t arena_bytes;   /* size of the arena */
  size_t peak_bytes;    /* most arena bytes held by slots at once */
} tat_service_stats;

/* Defaults: 8 GiB budget, max_batch 32, graphs on, autotune off, one graph per flush. */
tat_status tat_service_config_default(tat_service_config* cfg);

/* Creates a service on the current device and allocates its arena.
 * TAT_ERR_OOM if the arena cannot be allocated. */
tat_status tat_service_create(tat_service_t* svc, const tat_service_config* cfg);
tat_status tat_service_destroy(tat_service_t svc);

/* Queues op(in) -> out for the problem `desc` (validated on the host; the
 * plan is built at the first flush that needs it).  in/out sizes: n*n floats
 * for images, n_det*n_t floats for data (TAT_OP_PAIR: both images).  *id receives the request's index
 * (0, 1, 2, ... in submission order). */
tat_status tat_service_submit(tat_service_t svc, const tat_plan_desc* desc, tat_op op, const float* in,
                              float* out, long long* id);

/* Launches every queued request (asynchronously) and returns. */
tat_status tat_service_flush(tat_service_t svc);

/* Waits for all launched work. */
tat_status tat_service_synchronize(tat_service_t svc);

/* Host time in ms from a request's submission to its completion, and its
 * status (TAT_ERR_INVALID_ARG if the id is unknown or it has not completed). */
tat_status tat_service_latency(tat_service_t svc, long long id, double* ms, tat_status* status);

tat_status tat_service_get_stats(tat_service_t svc, tat_service_stats* stats);

/* Times the launch shapes the kernels take at run time -- column strips of
 * 2, 4, 8, 16, 32 half-plane columns per CTA in the column stages and 1, 2, 4
 * row pairs per CTA in the row stages (those within the device limits), then,
 * for the best of those, column CTAs of 64, 128 and 384 threads (instead of 256; 64 and
 * 128 for the four-step column lengths only) with half, the same and twice its strip, then
 * row groups of 64 and 128 threads (instead of 256; lengths N <= 1024) with 1, 2
 * and 4 times its row pairs, the best shape with and without programmatic
 * dependent launch of the stages, the other pass order of the length-2M FFT of
 * the cosine and sine stages (tat_plan_set_fft_order) and the other column transforms
 * (tat_plan_set_column_split, where the split one applies; with half, the same and twice
 * the strip and, where a column stage then runs the four-step transform, column CTAs of
 * 64, 128, 256 and 384 threads) -- on
 * one A then one A* of `batch` images at f (device, batch*n*n floats, output
 * of A* written to f_out) with g (batch*n_det*n_t floats) and the workspace
 * for `batch`, and keeps the fastest for every later call on this plan.  The
 * shapes only regroup work: A* is unchanged bit for bit, A and A^-1 up to the
 * rounding of the FFT pass order (and both up to that of the column transform).  Synchronises `stream`.  *ms_best
 * (optional) receives the chosen shape's time for the pair, *strip,
 * *row_pairs, *cols_threads and *row_threads (optional) the chosen knobs
 * (tat_plan_get_fft_order reports the chosen pass order). */
tat_status tat_plan_autotune(tat_plan_t plan, int batch, float* f, float* g, float* f_out, void* workspace,
                             tat_stream_t stream, double* ms_best, int* strip, int* row_pairs, int* cols_threads,
                             int* row_threads);

/* Sets the same knobs directly (for instance to reuse shapes tuned earlier): `strip`
 * columns per column CTA, `row_pairs` per row CTA, `cols_threads` threads per column
 * CTA (a multiple of 32, at most 384 for the column lengths up to 4096 with a
 * compile-time schedule; below 256 only for the four-step column lengths 512 .. 4096),
 * `row_threads` threads per row pair (a multiple of 32 for the four-step lengths up to
 * 4096, else the plan's own; 0 keeps the current value).  TAT_ERR_UNSUPPORTED, with the
 * plan unchanged, for shapes outside the device or kernel limits.  Results do not depend
 * on the shapes (A* bit for bit: its scatter adds in a fixed order).  Host only. */
tat_status tat_plan_set_launch_shape(tat_plan_t plan, int strip, int row_pairs, int cols_threads, int row_threads);

/* Pass order of the length-2M FFT inside the cosine (A, A*) and sine (A^-1) stages: 0 runs
 * the radix-3 passes first, 1 the same passes in reverse (the tail radix first).  The
 * results agree to rounding.  tat_plan_autotune tries both and keeps the faster; these set
 * and read the order directly.  TAT_ERR_INVALID_ARG for an order other than 0 or 1. */
tat_status tat_plan_set_fft_order(tat_plan_t plan, int order);
tat_status tat_plan_get_fft_order(tat_plan_t plan, int* order);

/* Column transform of the column stages of A and A* (Algorithm 1 step 2 and its transpose)
 * at N = 512 RB (RB = 1, 2, 4, 8, 16) with n <= 512 (n <= 1024 at N = 8192).  The split
 * transform divides each length-N column DFT into RB 512-point DFTs, one per warp of a CTA
 * of RB warps (the column's rows are zero from n on, so bin q = k1 + RB k2 takes only the
 * 512-point DFT k2 of the rows twiddled by w_N^(m k1), at N = 8192 with the rows m + 512
 * folded onto m); the other runs the four-step transform in CTA-wide passes.  `mask` bit 0
 * selects the split transform for the column stage of A, bit 1 for that of A* (0 .. 3;
 * A^-1's column stage keeps the four-step transform).  Plan defaults: 3 at
 * N = 1024 .. 4096, 1 at N = 512, 2 at N = 8192, 0 where the split transform does not
 * apply (there the setting is kept and has no effect); tat_plan_autotune tries the other
 * values.  The transforms agree to rounding (each is deterministic bit for bit on its
 * own).  TAT_ERR_INVALID_ARG outside 0 .. 3. */
tat_status tat_plan_set_column_split(tat_plan_t plan, int mask);
tat_status tat_plan_get_column_split(tat_plan_t plan, int* mask);

#ifdef __cplusplus
}
#endif
#endif /* TAT_SERVICE_H_ */
