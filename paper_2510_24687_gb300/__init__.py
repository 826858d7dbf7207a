"""GB300-native fast forward operator A and adjoint A* for photoacoustic /
thermoacoustic tomography with detectors on a circle (Hauptmann, Kunyansky,
Poimala, arXiv 2510.24687, Algorithms 1 and 2).

The operators run as hand-written CUDA kernels for sm_103a inside libtat.so,
whose C ABI is declared in include/tat.h; this package is its thin binding.
"""
from .binding import (TatError, TatOperator, header_symbols, load, tat_adjoint, tat_adjoint_batched,
                      tat_debug_adjoint_batched_timed, tat_debug_bessel, tat_debug_forward_batched_timed,
                      tat_debug_low_mode_rule, tat_debug_stencils, tat_forward,
                      tat_forward_batched, tat_forward_noalloc, tat_plan_create, tat_plan_create_ex, tat_plan_desc,
                      tat_plan_desc_default, tat_plan_destroy, tat_plan_get_info, tat_plan_info,
                      tat_plan_query, tat_status_string, tat_workspace_size)

__all__ = ["TatError", "TatOperator", "header_symbols", "load", "tat_adjoint", "tat_adjoint_batched",
           "tat_debug_adjoint_batched_timed", "tat_debug_bessel", "tat_debug_forward_batched_timed",
           "tat_debug_low_mode_rule", "tat_debug_stencils", "tat_forward",
           "tat_forward_batched", "tat_forward_noalloc", "tat_plan_create", "tat_plan_create_ex", "tat_plan_desc",
           "tat_plan_desc_default", "tat_plan_destroy", "tat_plan_get_info", "tat_plan_info", "tat_plan_query",
           "tat_status_string", "tat_workspace_size"]

from . import autograd, lpd, solvers  # noqa: E402
from .binding import (tat_adam, tat_conv_in_bwd, tat_conv_in_bwd_data, tat_conv_in_bwd_weights, tat_conv_in_fwd,  # noqa: E402
                      tat_conv_mid_bwd_data, tat_conv_mid_bwd_weights, tat_conv_mid_fwd, tat_conv_out_bwd,
                      tat_conv_out_fwd, tat_fill, tat_lpd_check, tat_lpd_scratch_floats, tat_lpd_timeout_probe, tat_mse, tat_to_bf16)
from .autograd import A, Astar  # noqa: E402
from .solvers import TatSolver, nnls_unrolled, pdhg_steps, power_norm_sq, tv_unrolled  # noqa: E402
from .binding import tat_debug_inverse_batched_timed, tat_inverse, tat_inverse_batched  # noqa: E402
from .binding import (TatService, tat_plan_autotune, tat_plan_get_fft_order, tat_plan_set_fft_order,  # noqa: E402
                      tat_plan_get_column_split, tat_plan_set_column_split,
                      tat_plan_set_launch_shape, tat_service_config_default, tat_service_create,
                      tat_service_destroy, tat_service_flush, tat_service_get_stats, tat_service_latency,
                      tat_service_submit, tat_service_synchronize)
from .binding import (tat_axpby_clamp, tat_axpby_clamp_backward, tat_pd_dual_data, tat_tv_dual,  # noqa: E402
                      tat_tv_dual_backward, tat_tv_primal, tat_tv_primal_backward)

__all__ += ["lpd", "tat_adam", "tat_conv_in_bwd", "tat_conv_in_bwd_data", "tat_conv_in_bwd_weights", "tat_conv_in_fwd",
            "tat_conv_mid_bwd_data", "tat_conv_mid_bwd_weights", "tat_conv_mid_fwd", "tat_conv_out_bwd",
            "tat_conv_out_fwd", "tat_fill", "tat_lpd_check", "tat_lpd_scratch_floats", "tat_lpd_timeout_probe", "tat_mse", "tat_to_bf16", "TatService", "tat_plan_autotune", "tat_plan_get_fft_order", "tat_plan_set_fft_order", "tat_plan_get_column_split", "tat_plan_set_column_split", "tat_plan_set_launch_shape", "tat_service_config_default", "tat_service_create",
            "tat_service_destroy", "tat_service_flush", "tat_service_get_stats", "tat_service_latency",
            "tat_service_submit", "tat_service_synchronize", "tat_inverse", "tat_inverse_batched", "tat_debug_inverse_batched_timed", "autograd", "solvers", "A", "Astar", "TatSolver", "nnls_unrolled", "pdhg_steps", "power_norm_sq",
            "tv_unrolled", "tat_axpby_clamp", "tat_axpby_clamp_backward", "tat_pd_dual_data", "tat_tv_dual",
            "tat_tv_dual_backward", "tat_tv_primal", "tat_tv_primal_backward"]
