// C ABI of the fast circular-geometry operators; see include/tat.h.
#include <cmath>
#include <cstdint>
#include <new>

#include "plan.hpp"
#include "tat_debug.h"

namespace {

constexpr double kTwoPi = 6.28318530717958647692528676655900577;

tat_status check_pointers(const void* a, const void* b, const void* ws) {
  if (!a || !b || !ws) return TAT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return TAT_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(a) % 4 || reinterpret_cast<uintptr_t>(b) % 4) return TAT_ERR_INVALID_ARG;
  return TAT_OK;
}

tat_status check_device(const tat_plan_s* P) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TAT_ERR_CUDA;
  }
  return dev == P->device ? TAT_OK : TAT_ERR_INVALID_ARG;
}

}  // namespace

extern "C" {

tat_status tat_plan_desc_default(tat_plan_desc* d, int n, int n_det, int n_t, double c, double R, double T) {
  if (!d) return TAT_ERR_INVALID_ARG;
  d->n = n;
  d->n_det = n_det;
  d->n_t = n_t;
  d->c = c;
  d->R = R;
  d->T = T;
  d->support_radius = 0.98;
  d->arc_begin = 0.0;
  d->arc_len = kTwoPi;
  d->n_phi = 0;
  d->pad_L = 0.0;
  d->low_mode_quadrature = 1;
  return TAT_OK;
}

tat_status tat_plan_query(const tat_plan_desc* desc, tat_plan_info* info) {
  if (!desc || !info) return TAT_ERR_INVALID_ARG;
  tat::Grids G;
  const tat_status s = tat::derive_grids(*desc, &G);
  if (s != TAT_OK) return s;
  tat::fill_info(G, info);
  return TAT_OK;
}

tat_status tat_plan_create_ex(tat_plan_t* plan, const tat_plan_desc* desc) {
  if (!plan) return TAT_ERR_INVALID_ARG;
  *plan = nullptr;
  if (!desc) return TAT_ERR_INVALID_ARG;
  {
    tat_plan_info probe;
    const tat_status q = tat_plan_query(desc, &probe);  // argument errors before any CUDA call
    if (q != TAT_OK) return q;
  }
  tat_plan_s* P = new (std::nothrow) tat_plan_s();
  if (!P) return TAT_ERR_OOM;
  if (cudaGetDevice(&P->device) != cudaSuccess) {
    cudaGetLastError();
    delete P;
    return TAT_ERR_CUDA;
  }
  tat_status s = tat::build_plan(*desc, P);
  if (s == TAT_OK) s = tat::validate_shapes(P);
  if (s == TAT_OK) s = tat::configure_kernels();
  if (s != TAT_OK) {
    tat::free_plan(P);
    delete P;
    return s;
  }
  *plan = P;
  return TAT_OK;
}

tat_status tat_plan_create(tat_plan_t* plan, int n, int n_det, int n_t, double c, double R, double T) {
  tat_plan_desc d;
  tat_plan_desc_default(&d, n, n_det, n_t, c, R, T);
  return tat_plan_create_ex(plan, &d);
}

tat_status tat_plan_destroy(tat_plan_t plan) {
  if (!plan) return TAT_ERR_INVALID_ARG;
  tat::free_plan(plan);
  delete plan;
  return TAT_OK;
}

tat_status tat_plan_get_info(tat_plan_t plan, tat_plan_info* info) {
  if (!plan || !info) return TAT_ERR_INVALID_ARG;
  *info = plan->info;
  return TAT_OK;
}

size_t tat_workspace_size(tat_plan_t plan, int batch) {
  if (!plan || batch < 1) return 0;
  return (size_t)batch * (plan->ws_x + plan->ws_y) * sizeof(float2);
}

tat_status tat_forward_batched(tat_plan_t plan, int batch, const float* f, long long f_stride, float* g,
                               long long g_stride, void* workspace, tat_stream_t stream) {
  if (!plan || batch < 1) return TAT_ERR_INVALID_ARG;
  const tat::DevPlan& d = plan->d;
  if (f_stride < (long long)d.n * d.n || g_stride < (long long)d.n_det * d.n_t) return TAT_ERR_INVALID_ARG;
  tat_status s = check_pointers(f, g, workspace);
  if (s == TAT_OK) s = check_device(plan);
  if (s != TAT_OK) return s;
  return tat::launch_forward(plan, batch, f, f_stride, g, g_stride, workspace, static_cast<cudaStream_t>(stream));
}

tat_status tat_adjoint_batched(tat_plan_t plan, int batch, const float* g, long long g_stride, float* f,
                               long long f_stride, void* workspace, tat_stream_t stream) {
  if (!plan || batch < 1) return TAT_ERR_INVALID_ARG;
  const tat::DevPlan& d = plan->d;
  if (f_stride < (long long)d.n * d.n || g_stride < (long long)d.n_det * d.n_t) return TAT_ERR_INVALID_ARG;
  tat_status s = check_pointers(g, f, workspace);
  if (s == TAT_OK) s = check_device(plan);
  if (s != TAT_OK) return s;
  return tat::launch_adjoint(plan, batch, g, g_stride, f, f_stride, workspace, static_cast<cudaStream_t>(stream));
}

tat_status tat_forward(tat_plan_t plan, const float* f, float* g, void* workspace, tat_stream_t stream) {
  if (!plan) return TAT_ERR_INVALID_ARG;
  return tat_forward_batched(plan, 1, f, (long long)plan->d.n * plan->d.n, g,
                             (long long)plan->d.n_det * plan->d.n_t, workspace, stream);
}

tat_status tat_adjoint(tat_plan_t plan, const float* g, float* f, void* workspace, tat_stream_t stream) {
  if (!plan) return TAT_ERR_INVALID_ARG;
  return tat_adjoint_batched(plan, 1, g, (long long)plan->d.n_det * plan->d.n_t, f,
                             (long long)plan->d.n * plan->d.n, workspace, stream);
}

tat_status tat_inverse_batched(tat_plan_t plan, int batch, const float* g, long long g_stride, float* f,
                               long long f_stride, void* workspace, tat_stream_t stream) {
  if (!plan || batch < 1) return TAT_ERR_INVALID_ARG;
  const tat::DevPlan& d = plan->d;
  if (f_stride < (long long)d.n * d.n || g_stride < (long long)d.n_det * d.n_t) return TAT_ERR_INVALID_ARG;
  if (!d.inv_ok) return TAT_ERR_UNSUPPORTED;
  tat_status s = check_pointers(g, f, workspace);
  if (s == TAT_OK) s = check_device(plan);
  if (s != TAT_OK) return s;
  return tat::launch_inverse(plan, batch, g, g_stride, f, f_stride, workspace, static_cast<cudaStream_t>(stream));
}

tat_status tat_inverse(tat_plan_t plan, const float* g, float* f, void* workspace, tat_stream_t stream) {
  if (!plan) return TAT_ERR_INVALID_ARG;
  return tat_inverse_batched(plan, 1, g, (long long)plan->d.n_det * plan->d.n_t, f,
                             (long long)plan->d.n * plan->d.n, workspace, stream);
}

tat_status tat_debug_bessel(double x, int kmax, double* out) {
  if (!out || kmax < 0 || !(x >= 0)) return TAT_ERR_INVALID_ARG;
  tat::bessel_orders(x, kmax, out);
  return TAT_OK;
}

tat_status tat_debug_low_mode_rule(double* nodes, double* weights, int* count) {
  if (!count) return TAT_ERR_INVALID_ARG;
  if (nodes && weights && *count >= tat::kLowM) tat::low_mode_rule(nodes, weights);
  *count = tat::kLowM;
  return TAT_OK;
}

tat_status tat_debug_stencils(const tat_plan_desc* desc, int* ring, int* lp, int* i0, int* k0, double* a,
                              double* b, int count) {
  if (!desc || !ring || !lp || !i0 || !k0 || !a || !b || count < 0) return TAT_ERR_INVALID_ARG;
  tat::Grids G;
  const tat_status s = tat::derive_grids(*desc, &G);
  if (s != TAT_OK) return s;
  double lx[tat::kLowM], lw[tat::kLowM];
  if (G.low_on) tat::low_mode_rule(lx, lw);
  for (int e = 0; e < count; ++e) {
    const int r = ring[e];
    if (r < 1 || r > G.J + (G.low_on ? tat::kLowM : 0) || lp[e] < 0 || lp[e] >= G.n_phi / 2) return TAT_ERR_INVALID_ARG;
    const double lam = r <= G.J ? (double)r * G.dlam : lx[r - G.J - 1] * G.dlam;
    double c, sn;
    tat::cos_sin_2pi(lp[e] - G.n_phi / 4, G.n_phi, &c, &sn);
    const double u = lam * c / G.dxi, v = lam * sn / G.dxi;
    i0[e] = (int)std::floor(u);
    k0[e] = (int)std::floor(v);
    a[e] = u - std::floor(u);
    b[e] = v - std::floor(v);
  }
  return TAT_OK;
}

tat_status tat_debug_forward_batched_timed(tat_plan_t plan, int batch, const float* f, long long f_stride,
                                           float* g, long long g_stride, void* workspace, tat_stream_t stream,
                                           void* const* events) {
  if (!plan || batch < 1 || !events) return TAT_ERR_INVALID_ARG;
  const tat::DevPlan& d = plan->d;
  if (f_stride < (long long)d.n * d.n || g_stride < (long long)d.n_det * d.n_t) return TAT_ERR_INVALID_ARG;
  tat_status s = check_pointers(f, g, workspace);
  if (s == TAT_OK) s = check_device(plan);
  if (s != TAT_OK) return s;
  return tat::launch_forward(plan, batch, f, f_stride, g, g_stride, workspace, static_cast<cudaStream_t>(stream),
                             reinterpret_cast<cudaEvent_t const*>(events));
}

tat_status tat_debug_adjoint_batched_timed(tat_plan_t plan, int batch, const float* g, long long g_stride,
                                           float* f, long long f_stride, void* workspace, tat_stream_t stream,
                                           void* const* events) {
  if (!plan || batch < 1 || !events) return TAT_ERR_INVALID_ARG;
  const tat::DevPlan& d = plan->d;
  if (f_stride < (long long)d.n * d.n || g_stride < (long long)d.n_det * d.n_t) return TAT_ERR_INVALID_ARG;
  tat_status s = check_pointers(g, f, workspace);
  if (s == TAT_OK) s = check_device(plan);
  if (s != TAT_OK) return s;
  return tat::launch_adjoint(plan, batch, g, g_stride, f, f_stride, workspace, static_cast<cudaStream_t>(stream),
                             reinterpret_cast<cudaEvent_t const*>(events));
}

tat_status tat_debug_inverse_batched_timed(tat_plan_t plan, int batch, const float* g, long long g_stride,
                                           float* f, long long f_stride, void* workspace, tat_stream_t stream,
                                           void* const* events) {
  if (!plan || batch < 1 || !events) return TAT_ERR_INVALID_ARG;
  const tat::DevPlan& d = plan->d;
  if (f_stride < (long long)d.n * d.n || g_stride < (long long)d.n_det * d.n_t) return TAT_ERR_INVALID_ARG;
  if (!d.inv_ok) return TAT_ERR_UNSUPPORTED;
  tat_status s = check_pointers(g, f, workspace);
  if (s == TAT_OK) s = check_device(plan);
  if (s != TAT_OK) return s;
  return tat::launch_inverse(plan, batch, g, g_stride, f, f_stride, workspace, static_cast<cudaStream_t>(stream),
                             reinterpret_cast<cudaEvent_t const*>(events));
}

const char* tat_status_string(tat_status s) {
  switch (s) {
    case TAT_OK: return "ok";
    case TAT_ERR_INVALID_ARG: return "invalid argument";
    case TAT_ERR_UNSUPPORTED: return "unsupported configuration";
    case TAT_ERR_OOM: return "out of memory";
    case TAT_ERR_CUDA: return "CUDA error";
    case TAT_ERR_TIMEOUT: return "device wait timed out";
    case TAT_ERR_INTERNAL: return "internal error";
    default: return "unknown status";
  }
}

}  // extern "C"
