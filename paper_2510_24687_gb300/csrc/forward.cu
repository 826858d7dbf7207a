// Launcher of the forward operator A (Algorithm 1): five stream-ordered
// kernels per batch; see kernels.cuh for what each stage computes.
#include "launch.cuh"

namespace tat {

tat_status configure_kernels() { return TAT_OK; }

// Host-side check of every launch shape against the device limits.
tat_status validate_shapes(const tat_plan_s* Pl) {
  const Shapes s = shapes(Pl, 1);
  const size_t mx = 227 * 1024;
  const int blocks[] = {s.rows_block, s.cols_block, s.rings_block, s.modes_block, s.theta_block};
  const size_t smem[] = {s.rows_smem, s.cols_smem_f, s.cols_smem_a, s.rings_smem, s.modes_smem, s.theta_smem};
  for (int b : blocks)
    if (b < 32 || b > 1024 || b % 32) return TAT_ERR_UNSUPPORTED;
  if (s.cols_block > 512) return TAT_ERR_UNSUPPORTED;  // launch bound of the column kernels
  const int N = Pl->d.N;
  const bool ct = N == 256 || N == 512 || N == 1024 || N == 2048 || N == 4096 || N == 8192;
  if (ct && N <= 4096 && s.cols_block > 384) return TAT_ERR_UNSUPPORTED;
  // the Stockham column FFT runs on nt_N threads of the CTA; the four-step one on any multiple of 32
  const bool four = N == 512 || N == 1024 || N == 2048 || N == 4096 || N == 8192;
  if (!four && (s.cols_block < Pl->cfg.nt_N || s.cols_block < 256)) return TAT_ERR_UNSUPPORTED;
  // a row group runs the Stockham FFT on exactly nt_N threads; the four-step one on any multiple of 32
  if (four ? Pl->cfg.nt_rows % 32 != 0 : Pl->cfg.nt_rows != Pl->cfg.nt_N) return TAT_ERR_UNSUPPORTED;
  if (N == 8192 && s.rows_block > 512) return TAT_ERR_UNSUPPORTED;  // launch bound of the row kernels there
  for (size_t m : smem)
    if (m > mx) return TAT_ERR_UNSUPPORTED;
  if (Pl->cfg.t_tile % 2 || Pl->cfg.strip < 1 || Pl->cfg.rings_per_cta < 1) return TAT_ERR_INVALID_ARG;
  return TAT_OK;
}

tat_status launch_forward(const tat_plan_s* Pl, int batch, const float* f, long long fs, float* g, long long gs,
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
  dispatch_N(P.N, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value;
    ok &= ensure_smem<k_rows_fwd<L>>(dev) && ensure_smem<k_cols_fwd<L>>(dev);
    ok &= pdl_launch(c.pdl != 0, k_rows_fwd<L>, s.rows_grid, s.rows_block, s.rows_smem, st, P, f, fs, X, xs, c.rows_pairs, c.nt_rows) == cudaSuccess;
    stage_done();
    if constexpr (split_length(L)) {
      if (s.cols_split_f) {
        ok &= ensure_smem<k_cols_fwd_split<L>>(dev);
        ok &= pdl_launch(c.pdl != 0, k_cols_fwd_split<L>, s.cols_grid_f, s.cols_block_split, s.cols_smem_f, st, P, X, xs, Y, ys, c.strip, batch) == cudaSuccess;
      } else {
        ok &= pdl_launch(c.pdl != 0, k_cols_fwd<L>, s.cols_grid_f, s.cols_block, s.cols_smem_f, st, P, X, xs, Y, ys, c.strip, c.nt_N, batch) == cudaSuccess;
      }
    } else {
      ok &= pdl_launch(c.pdl != 0, k_cols_fwd<L>, s.cols_grid_f, s.cols_block, s.cols_smem_f, st, P, X, xs, Y, ys, c.strip, c.nt_N, batch) == cudaSuccess;
    }
    stage_done();
  });
  dispatch_ang(P.n_phi, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value;
    ok &= ensure_smem<k_rings_fwd<L>>(dev);
    ok &= pdl_launch(c.pdl != 0, k_rings_fwd<L>, s.rings_grid, s.rings_block, s.rings_smem, st, P, Y, ys, X, xs, c.rings_per_cta, c.nt_phi, s.ntiles) == cudaSuccess;
    stage_done();
  });
  dispatch_2M(2 * P.M, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value;
    dispatch_order(L > 0 ? c.order_2M : 0, [&](auto Vc) {
      constexpr int V = decltype(Vc)::value;
      ok &= ensure_smem<k_modes_fwd<L, V>>(dev);
      ok &= pdl_launch(c.pdl != 0, k_modes_fwd<L, V>, s.modes_grid, s.modes_block, s.modes_smem, st, P, X, xs, Y, ys, c.nt_2M) == cudaSuccess;
    });
    stage_done();
  });
  dispatch_ang(P.n_det, [&](auto Lc) {
    constexpr int L = decltype(Lc)::value;
    ok &= ensure_smem<k_theta_fwd<L>>(dev);
    ok &= pdl_launch(c.pdl != 0, k_theta_fwd<L>, s.theta_grid, s.theta_block, s.theta_smem, st, P, Y, ys, g, gs, c.t_tile, c.nt_det) == cudaSuccess;
    stage_done();
  });
  return check_launch(ok);
}

}  // namespace tat
