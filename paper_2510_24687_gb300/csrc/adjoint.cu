// Launcher of the adjoint A* (the stages of Algorithm 2 as the exact transpose
// of Algorithm 1): five stream-ordered kernels per batch, in reverse order.
#include "launch.cuh"

namespace tat {

tat_status launch_adjoint(const tat_plan_s* Pl, int batch, const float* g, long long gs, float* f, long long fs,
                          void* ws, cudaStream_t st, cudaEvent_t const* ev) {
  const DevPlan& P = Pl->d;
  const LaunchCfg& c = Pl->cfg;
  const Shapes s = shapes(Pl, batch);
  float2* X = static_cast<float2*>(ws);
  float2* Y = X + (size_t)batch * Pl->ws_x;
  const long long xs = (long long)Pl->ws_x, ys = (long long)Pl->ws_y;
  const int dev = Pl->device;
  bool ok = true;
  int mark = 0;
  auto stage_done = [&]() {
    if (ev) cudaEventRecord(ev[mark++], st);
  };
  stage_done();
  dispatch_ang(P.n_det, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value;
    ok &= ensure_smem<k_theta_adj<L>>(dev);
    ok &= pdl_launch(c.pdl != 0, k_theta_adj<L>, s.theta_grid, s.theta_block, s.theta_smem, st, P, g, gs, Y, ys, c.t_tile, c.nt_det) == cudaSuccess;
    stage_done();
  });
  dispatch_2M(2 * P.M, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value;
    dispatch_order(L > 0 ? c.order_2M : 0, [&](auto Vc) {
      constexpr int V = decltype(Vc)::value;
      ok &= ensure_smem<k_modes_adj<L, V>>(dev);
      ok &= pdl_launch(c.pdl != 0, k_modes_adj<L, V>, s.modes_grid, s.modes_block, s.modes_smem, st, P, Y, ys, X, xs, c.nt_2M) == cudaSuccess;
    });
    stage_done();
  });
  dispatch_ang(P.n_phi, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value;
    ok &= ensure_smem<k_rings_adj<L>>(dev);
    ok &= pdl_launch(c.pdl != 0, k_rings_adj<L>, s.rings_grid, s.rings_block, s.rings_smem, st, P, X, xs, Y, ys, c.rings_per_cta, c.nt_phi, s.ntiles) == cudaSuccess;
    stage_done();
  });
  dispatch_N(P.N, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value;
    ok &= ensure_smem<k_cols_adj<L>>(dev) && ensure_smem<k_rows_adj<L>>(dev);
    if constexpr (split_length(L)) {
      if (s.cols_split_a) {
        ok &= ensure_smem<k_cols_adj_split<L>>(dev);
        ok &= pdl_launch(c.pdl != 0, k_cols_adj_split<L>, s.cols_grid_a, s.cols_block_split, s.cols_smem_a, st, P, Y, ys, X, xs, c.strip, batch) == cudaSuccess;
      } else {
        ok &= pdl_launch(c.pdl != 0, k_cols_adj<L>, s.cols_grid_a, s.cols_block, s.cols_smem_a, st, P, Y, ys, X, xs, c.strip, c.nt_N, batch) == cudaSuccess;
      }
    } else {
      ok &= pdl_launch(c.pdl != 0, k_cols_adj<L>, s.cols_grid_a, s.cols_block, s.cols_smem_a, st, P, Y, ys, X, xs, c.strip, c.nt_N, batch) == cudaSuccess;
    }
    stage_done();
    ok &= pdl_launch(c.pdl != 0, k_rows_adj<L>, s.rows_grid, s.rows_block, s.rows_smem, st, P, X, xs, f, fs, c.rows_pairs, c.nt_rows) == cudaSuccess;
    stage_done();
  });
  return check_launch(ok);
}

}  // namespace tat
