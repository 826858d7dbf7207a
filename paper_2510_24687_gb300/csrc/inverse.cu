// Launcher of the approximate inverse A^{-1} (Algorithm 3, universal
// backprojection with the constant C of Eq. silly_integral): six
// stream-ordered kernels per batch on the grids of the adjoint; see
// kernels.cuh for what each stage computes.
#include "launch.cuh"

namespace tat {

tat_status launch_inverse(const tat_plan_s* Pl, int batch, const float* g, long long gs, float* f, long long fs,
                          void* ws, cudaStream_t st, cudaEvent_t const* ev) {
  const DevPlan& P = Pl->d;
  if (!P.inv_ok) return TAT_ERR_UNSUPPORTED;
  const LaunchCfg& c = Pl->cfg;
  const Shapes s = shapes(Pl, batch);
  float2* X = static_cast<float2*>(ws);
  float2* Y = X + (size_t)batch * Pl->ws_x;
  const long long xs = (long long)Pl->ws_x, ys = (long long)Pl->ws_y;
  // the per-image sum for C: element 0 of the image's Y region, as a float, and the row CTAs'
  // partial sums after it (the polar samples there are consumed by the column stage)
  float* acc = reinterpret_cast<float*>(Y);
  const long long accs = 2 * ys;
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
      ok &= ensure_smem<k_modes_inv<L, V>>(dev);
      ok &= pdl_launch(c.pdl != 0, k_modes_inv<L, V>, s.modes_grid, s.modes_block, s.modes_smem, st, P, Y, ys, X, xs, c.nt_2M) == cudaSuccess;
    });
    stage_done();
  });
  dispatch_ang(P.n_phi, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value;
    ok &= ensure_smem<k_rings_adj<L, true>>(dev);
    const dim3 grid(s.ntiles, batch);
    ok &= pdl_launch(c.pdl != 0, k_rings_adj<L, true>, grid, s.rings_block, s.rings_smem, st, P, X, xs, Y, ys, c.rings_per_cta, c.nt_phi, s.ntiles) == cudaSuccess;
    stage_done();
  });
  dispatch_N(P.N, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value;
    ok &= ensure_smem<k_cols_inv<L>>(dev) && ensure_smem<k_rows_inv<L>>(dev);
    ok &= pdl_launch(c.pdl != 0, k_cols_inv<L>, s.cols_grid_i, s.cols_block_i, s.cols_smem_i, st, P, Y, ys, X, xs, s.strip_i, c.nt_N, batch) == cudaSuccess;
    stage_done();
    ok &= pdl_launch(c.pdl != 0, k_rows_inv<L>, s.rows_grid, s.rows_block, s.rows_smem, st, P, X, xs, f, fs, acc, accs, c.rows_pairs, c.nt_rows) == cudaSuccess;
    stage_done();
  });
  {
    const long long count = (long long)batch * P.n * P.n;
    const int blocks = (int)std::min<long long>((count + 255) / 256, 152LL * 8);
    ok &= pdl_launch(c.pdl != 0, k_inv_sum, batch, 256, 0, st, (int)s.rows_grid.x, acc, accs) == cudaSuccess;
    ok &= pdl_launch(c.pdl != 0, k_inv_finish, blocks, 256, 0, st, P, batch, acc, accs, f, fs) == cudaSuccess;
    stage_done();
  }
  return check_launch(ok);
}

}  // namespace tat
