"""ctypes binding of libtat (include/tat.h, include/tat_debug.h, include/tat_solvers.h,
include/tat_service.h).

Argument marshalling only: every step of A and A* runs in the CUDA kernels of
libtat.  Functions keep the C names.  Device buffers are passed as integer
addresses (``tensor.data_ptr()``); ``TatOperator`` wraps a plan together with
torch-allocated outputs and workspace for convenience.  There is no CPU
fallback: if libtat.so is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import re

from ._build import LIB, ROOT

TAT_OK = 0
_STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported configuration", 3: "out of memory",
           4: "CUDA error", 5: "device wait timed out", 6: "internal error"}


class TatError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {_STATUS.get(status, 'unknown status')} (status {status})")
        self.status = status


class tat_plan_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("n_det", ctypes.c_int), ("n_t", ctypes.c_int),
                ("c", ctypes.c_double), ("R", ctypes.c_double), ("T", ctypes.c_double),
                ("support_radius", ctypes.c_double), ("arc_begin", ctypes.c_double),
                ("arc_len", ctypes.c_double), ("n_phi", ctypes.c_int), ("pad_L", ctypes.c_double),
                ("low_mode_quadrature", ctypes.c_int)]


class tat_plan_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("J", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("K", ctypes.c_int), ("n_low", ctypes.c_int), ("n_points", ctypes.c_int),
                ("h", ctypes.c_double), ("dt", ctypes.c_double), ("dlam", ctypes.c_double),
                ("dxi", ctypes.c_double), ("lam_c", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class tat_service_config(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_size_t), ("max_batch", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("autotune", ctypes.c_int), ("one_graph", ctypes.c_int)]


class tat_service_stats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("launches", ctypes.c_longlong),
                ("graph_launches", ctypes.c_longlong), ("flush_graphs", ctypes.c_longlong),
                ("evictions", ctypes.c_longlong), ("plans", ctypes.c_int),
                ("slots", ctypes.c_int), ("arena_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


TAT_OP_FORWARD, TAT_OP_ADJOINT, TAT_OP_INVERSE, TAT_OP_PAIR = 0, 1, 2, 3

_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_LL = ctypes.c_longlong
_D = ctypes.c_double
_F = ctypes.c_float


def load() -> ctypes.CDLL:
    """Loads libtat.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"{LIB} is missing: run __graft_entry__.build() (there is no CPU fallback)")
    lib = ctypes.CDLL(LIB)
    sig = {
        "tat_plan_desc_default": (_I, [ctypes.POINTER(tat_plan_desc), _I, _I, _I, _D, _D, _D]),
        "tat_plan_query": (_I, [ctypes.POINTER(tat_plan_desc), ctypes.POINTER(tat_plan_info)]),
        "tat_plan_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, _D, _D, _D]),
        "tat_plan_create_ex": (_I, [ctypes.POINTER(_P), ctypes.POINTER(tat_plan_desc)]),
        "tat_plan_destroy": (_I, [_P]),
        "tat_plan_get_info": (_I, [_P, ctypes.POINTER(tat_plan_info)]),
        "tat_workspace_size": (ctypes.c_size_t, [_P, _I]),
        "tat_forward": (_I, [_P, _P, _P, _P, _P]),
        "tat_adjoint": (_I, [_P, _P, _P, _P, _P]),
        "tat_forward_batched": (_I, [_P, _I, _P, _LL, _P, _LL, _P, _P]),
        "tat_adjoint_batched": (_I, [_P, _I, _P, _LL, _P, _LL, _P, _P]),
        "tat_status_string": (ctypes.c_char_p, [_I]),
        "tat_debug_bessel": (_I, [_D, _I, ctypes.POINTER(_D)]),
        "tat_debug_low_mode_rule": (_I, [ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I)]),
        "tat_debug_stencils": (_I, [ctypes.POINTER(tat_plan_desc), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                    ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_D),
                                    ctypes.POINTER(_D), _I]),
        "tat_forward_noalloc": (_I, [_P, _P, _P, _P]),
        "tat_inverse": (_I, [_P, _P, _P, _P, _P]),
        "tat_inverse_batched": (_I, [_P, _I, _P, _LL, _P, _LL, _P, _P]),
        "tat_debug_inverse_batched_timed": (_I, [_P, _I, _P, _LL, _P, _LL, _P, _P, ctypes.POINTER(_P)]),
        "tat_debug_forward_batched_timed": (_I, [_P, _I, _P, _LL, _P, _LL, _P, _P, ctypes.POINTER(_P)]),
        "tat_debug_adjoint_batched_timed": (_I, [_P, _I, _P, _LL, _P, _LL, _P, _P, ctypes.POINTER(_P)]),
        "tat_service_config_default": (_I, [ctypes.POINTER(tat_service_config)]),
        "tat_service_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(tat_service_config)]),
        "tat_service_destroy": (_I, [_P]),
        "tat_service_submit": (_I, [_P, ctypes.POINTER(tat_plan_desc), _I, _P, _P, ctypes.POINTER(_LL)]),
        "tat_service_flush": (_I, [_P]),
        "tat_service_synchronize": (_I, [_P]),
        "tat_service_latency": (_I, [_P, _LL, ctypes.POINTER(_D), ctypes.POINTER(_I)]),
        "tat_service_get_stats": (_I, [_P, ctypes.POINTER(tat_service_stats)]),
        "tat_plan_autotune": (_I, [_P, _I, _P, _P, _P, _P, _P, ctypes.POINTER(_D), ctypes.POINTER(_I),
                                   ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
        "tat_plan_set_launch_shape": (_I, [_P, _I, _I, _I, _I]),
        "tat_plan_set_fft_order": (_I, [_P, _I]),
        "tat_plan_get_fft_order": (_I, [_P, ctypes.POINTER(_I)]),
        "tat_plan_set_column_split": (_I, [_P, _I]),
        "tat_plan_get_column_split": (_I, [_P, ctypes.POINTER(_I)]),
        "tat_lpd_scratch_floats": (ctypes.c_size_t, [_I, _I, _I]),
        "tat_conv_in_fwd": (_I, [_I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P]),
        "tat_conv_in_bwd_data": (_I, [_I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _I, _P]),
        "tat_conv_in_bwd_weights": (_I, [_I, _I, _I, _I, _P, _P, _P, _P, _P, _P, ctypes.c_size_t, _P, _P, _P]),
        "tat_conv_in_bwd": (_I, [_I, _I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _P, ctypes.c_size_t, _P, _P,
                                 _P]),
        "tat_conv_mid_fwd": (_I, [_I, _I, _I, _P, _P, _P, _P, _P]),
        "tat_conv_mid_bwd_data": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P]),
        "tat_conv_mid_bwd_weights": (_I, [_I, _I, _I, _P, _P, _P, _P, ctypes.c_size_t, _P, _P, _P]),
        "tat_conv_out_fwd": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P]),
        "tat_conv_out_bwd": (_I, [_I, _I, _I, _P, _P, _P, _I, _P, _P, ctypes.c_size_t, _P, _P, _P]),
        "tat_adam": (_I, [_LL, _F, _F, _F, _F, _I, _P, _P, _P, _P, _P, _P]),
        "tat_to_bf16": (_I, [_LL, _P, _P, _P]),
        "tat_fill": (_I, [_LL, _F, _P, _P]),
        "tat_lpd_check": (_I, []),
        "tat_lpd_timeout_probe": (_I, [_I, _P, _P]),
        "tat_mse": (_I, [_LL, _P, _P, _F, _P, _P, _P]),
        "tat_axpby_clamp": (_I, [_LL, _F, _P, _F, _P, _F, _P, _LL, _P, _P]),
        "tat_axpby_clamp_backward": (_I, [_LL, _P, _F, _P, _LL, _P, _F, _P, _F, _P, _P]),
        "tat_pd_dual_data": (_I, [_LL, _F, _P, _P, _P, _P, _P]),
        "tat_tv_dual": (_I, [_I, _I, _F, _F, _F, _P, _P, _P, _P]),
        "tat_tv_dual_backward": (_I, [_I, _I, _F, _F, _F, _P, _P, _P, _P, _P, _P]),
        "tat_tv_primal": (_I, [_I, _I, _F, _F, _P, _P, _P, _P, _P, _P, _P]),
        "tat_tv_primal_backward": (_I, [_I, _I, _F, _F, _P, _P, _P, _P, _P, _P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_symbols():
    """Function names declared in include/*.h (for the ABI export test)."""
    names = []
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            txt = open(os.path.join(inc, h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tat_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def _check(status: int, what: str):
    if status != TAT_OK:
        raise TatError(status, what)


# ------------------------------------------------------------------ C names

def tat_plan_desc_default(n, n_det, n_t, c=1.0, R=1.0, T=2.0) -> tat_plan_desc:
    d = tat_plan_desc()
    _check(load().tat_plan_desc_default(ctypes.byref(d), n, n_det, n_t, c, R, T), "tat_plan_desc_default")
    return d


def tat_plan_query(desc: tat_plan_desc) -> dict:
    info = tat_plan_info()
    _check(load().tat_plan_query(ctypes.byref(desc), ctypes.byref(info)), "tat_plan_query")
    return info.as_dict()


def tat_plan_create(n, n_det, n_t, c=1.0, R=1.0, T=2.0) -> int:
    h = _P()
    _check(load().tat_plan_create(ctypes.byref(h), n, n_det, n_t, c, R, T), "tat_plan_create")
    return h.value


def tat_plan_create_ex(desc: tat_plan_desc) -> int:
    h = _P()
    _check(load().tat_plan_create_ex(ctypes.byref(h), ctypes.byref(desc)), "tat_plan_create_ex")
    return h.value


def tat_plan_destroy(plan: int):
    _check(load().tat_plan_destroy(plan), "tat_plan_destroy")


def tat_plan_get_info(plan: int) -> dict:
    info = tat_plan_info()
    _check(load().tat_plan_get_info(plan, ctypes.byref(info)), "tat_plan_get_info")
    return info.as_dict()


def tat_workspace_size(plan: int, batch: int = 1) -> int:
    return int(load().tat_workspace_size(plan, batch))


def tat_forward(plan, f_ptr, g_ptr, ws_ptr, stream=0):
    _check(load().tat_forward(plan, f_ptr, g_ptr, ws_ptr, stream or None), "tat_forward")


def tat_adjoint(plan, g_ptr, f_ptr, ws_ptr, stream=0):
    _check(load().tat_adjoint(plan, g_ptr, f_ptr, ws_ptr, stream or None), "tat_adjoint")


def tat_inverse(plan, g_ptr, f_ptr, ws_ptr, stream=0):
    _check(load().tat_inverse(plan, g_ptr, f_ptr, ws_ptr, stream or None), "tat_inverse")


def tat_inverse_batched(plan, batch, g_ptr, g_stride, f_ptr, f_stride, ws_ptr, stream=0):
    _check(load().tat_inverse_batched(plan, batch, g_ptr, g_stride, f_ptr, f_stride, ws_ptr, stream or None),
           "tat_inverse_batched")


def tat_debug_inverse_batched_timed(plan, batch, g_ptr, g_stride, f_ptr, f_stride, ws_ptr, stream, events):
    """events: 7 raw cudaEvent_t handles."""
    _check(load().tat_debug_inverse_batched_timed(plan, batch, g_ptr, g_stride, f_ptr, f_stride, ws_ptr,
                                                  stream or None, _events(events)), "tat_debug_inverse_batched_timed")


def tat_forward_noalloc(plan, f_ptr, g_ptr, stream=0):
    """A f for one image using the library's static scratch buffer (no workspace, no allocation)."""
    _check(load().tat_forward_noalloc(plan, f_ptr, g_ptr, stream or None), "tat_forward_noalloc")


def tat_forward_batched(plan, batch, f_ptr, f_stride, g_ptr, g_stride, ws_ptr, stream=0):
    _check(load().tat_forward_batched(plan, batch, f_ptr, f_stride, g_ptr, g_stride, ws_ptr, stream or None),
           "tat_forward_batched")


def tat_adjoint_batched(plan, batch, g_ptr, g_stride, f_ptr, f_stride, ws_ptr, stream=0):
    _check(load().tat_adjoint_batched(plan, batch, g_ptr, g_stride, f_ptr, f_stride, ws_ptr, stream or None),
           "tat_adjoint_batched")


def _events(evs):
    arr = (_P * len(evs))(*evs)
    return arr


def tat_debug_forward_batched_timed(plan, batch, f_ptr, f_stride, g_ptr, g_stride, ws_ptr, stream, events):
    """events: 6 raw cudaEvent_t handles (e.g. torch.cuda.Event(...).cuda_event after one record())."""
    _check(load().tat_debug_forward_batched_timed(plan, batch, f_ptr, f_stride, g_ptr, g_stride, ws_ptr,
                                                  stream or None, _events(events)), "tat_debug_forward_batched_timed")


def tat_debug_adjoint_batched_timed(plan, batch, g_ptr, g_stride, f_ptr, f_stride, ws_ptr, stream, events):
    _check(load().tat_debug_adjoint_batched_timed(plan, batch, g_ptr, g_stride, f_ptr, f_stride, ws_ptr,
                                                  stream or None, _events(events)), "tat_debug_adjoint_batched_timed")


def tat_axpby_clamp(count, a, x_ptr, b, y_ptr, lo, mask_ptr, mask_period, out_ptr, stream=0):
    """out = mask * max(lo, a*x + b*y); y_ptr / mask_ptr may be 0."""
    _check(load().tat_axpby_clamp(count, a, x_ptr, b, y_ptr or None, lo, mask_ptr or None, mask_period, out_ptr,
                                  stream or None), "tat_axpby_clamp")


def tat_axpby_clamp_backward(count, out_ptr, lo, mask_ptr, mask_period, grad_out_ptr, a, grad_x_ptr, b, grad_y_ptr,
                             stream=0):
    """G = mask [out > lo] grad_out; grad_x = a G, grad_y = b G (either pointer may be 0)."""
    _check(load().tat_axpby_clamp_backward(count, out_ptr, lo, mask_ptr or None, mask_period, grad_out_ptr, a,
                                           grad_x_ptr or None, b, grad_y_ptr or None, stream or None),
           "tat_axpby_clamp_backward")


def tat_pd_dual_data(count, sigma, Af_ptr, g_ptr, q_in_ptr, q_out_ptr, stream=0):
    """q_out = (q_in + sigma (Af - g)) / (1 + sigma)."""
    _check(load().tat_pd_dual_data(count, sigma, Af_ptr, g_ptr, q_in_ptr, q_out_ptr, stream or None),
           "tat_pd_dual_data")


def tat_tv_dual(batch, n, h_eff, sigma, bound, fbar_ptr, p_in_ptr, p_out_ptr, stream=0):
    """p_out = proj_{|p|<=bound}(p_in + sigma grad_h fbar)."""
    _check(load().tat_tv_dual(batch, n, h_eff, sigma, bound, fbar_ptr, p_in_ptr, p_out_ptr, stream or None),
           "tat_tv_dual")


def tat_tv_dual_backward(batch, n, h_eff, sigma, bound, fbar_ptr, p_in_ptr, grad_p_out_ptr, grad_p_in_ptr,
                         grad_fbar_ptr, stream=0):
    _check(load().tat_tv_dual_backward(batch, n, h_eff, sigma, bound, fbar_ptr, p_in_ptr, grad_p_out_ptr,
                                       grad_p_in_ptr, grad_fbar_ptr or None, stream or None), "tat_tv_dual_backward")


def tat_tv_primal(batch, n, h_eff, tau, Asq_ptr, p_ptr, mask_ptr, f_in_ptr, f_out_ptr, fbar_ptr, stream=0):
    """f_out = mask max(0, f_in - tau (Asq - div_h p)); fbar = 2 f_out - f_in."""
    _check(load().tat_tv_primal(batch, n, h_eff, tau, Asq_ptr, p_ptr, mask_ptr or None, f_in_ptr, f_out_ptr,
                                fbar_ptr, stream or None), "tat_tv_primal")


def tat_tv_primal_backward(batch, n, h_eff, tau, f_out_ptr, mask_ptr, grad_f_out_ptr, grad_fbar_ptr, grad_f_in_ptr,
                           grad_Asq_ptr, grad_p_ptr, stream=0):
    _check(load().tat_tv_primal_backward(batch, n, h_eff, tau, f_out_ptr, mask_ptr or None, grad_f_out_ptr or None,
                                         grad_fbar_ptr or None, grad_f_in_ptr or None, grad_Asq_ptr or None,
                                         grad_p_ptr or None, stream or None), "tat_tv_primal_backward")


def tat_plan_set_launch_shape(plan, strip, row_pairs, cols_threads, row_threads=0):
    _check(load().tat_plan_set_launch_shape(plan, strip, row_pairs, cols_threads, row_threads),
           "tat_plan_set_launch_shape")


def tat_plan_set_fft_order(plan, order):
    """Pass order (0 or 1) of the length-2M FFT of the cosine and sine stages."""
    _check(load().tat_plan_set_fft_order(plan, order), "tat_plan_set_fft_order")


def tat_plan_get_fft_order(plan):
    o = _I()
    _check(load().tat_plan_get_fft_order(plan, ctypes.byref(o)), "tat_plan_get_fft_order")
    return o.value


def tat_plan_set_column_split(plan, mask):
    """Column transforms at N = 512 RB: bit 0 (forward) / bit 1 (adjoint) set: RB warp-level
    512-point DFTs; clear: the four-step transform."""
    _check(load().tat_plan_set_column_split(plan, int(mask)), "tat_plan_set_column_split")


def tat_plan_get_column_split(plan):
    o = _I()
    _check(load().tat_plan_get_column_split(plan, ctypes.byref(o)), "tat_plan_get_column_split")
    return o.value


def tat_plan_autotune(plan, batch, f_ptr, g_ptr, f_out_ptr, ws_ptr, stream=0):
    """Times the runtime launch shapes on one A + A* of `batch` images; returns
    (ms, strip, row_pairs, cols_threads, row_threads)."""
    ms, strip, rp, ct, rt = _D(0), _I(0), _I(0), _I(0), _I(0)
    _check(load().tat_plan_autotune(plan, batch, f_ptr, g_ptr, f_out_ptr, ws_ptr, stream or None, ctypes.byref(ms),
                                    ctypes.byref(strip), ctypes.byref(rp), ctypes.byref(ct), ctypes.byref(rt)),
           "tat_plan_autotune")
    return ms.value, strip.value, rp.value, ct.value, rt.value


def tat_service_config_default() -> tat_service_config:
    c = tat_service_config()
    _check(load().tat_service_config_default(ctypes.byref(c)), "tat_service_config_default")
    return c


def tat_service_create(cfg: tat_service_config) -> int:
    h = _P()
    _check(load().tat_service_create(ctypes.byref(h), ctypes.byref(cfg)), "tat_service_create")
    return h.value


def tat_service_destroy(svc):
    _check(load().tat_service_destroy(svc), "tat_service_destroy")


def tat_service_submit(svc, desc: tat_plan_desc, op: int, in_ptr, out_ptr) -> int:
    rid = _LL(0)
    _check(load().tat_service_submit(svc, ctypes.byref(desc), op, in_ptr, out_ptr, ctypes.byref(rid)),
           "tat_service_submit")
    return rid.value


def tat_service_flush(svc):
    _check(load().tat_service_flush(svc), "tat_service_flush")


def tat_service_synchronize(svc):
    _check(load().tat_service_synchronize(svc), "tat_service_synchronize")


def tat_service_latency(svc, rid):
    ms, st = _D(0), _I(0)
    _check(load().tat_service_latency(svc, rid, ctypes.byref(ms), ctypes.byref(st)), "tat_service_latency")
    return ms.value, st.value


def tat_service_get_stats(svc) -> dict:
    st = tat_service_stats()
    _check(load().tat_service_get_stats(svc, ctypes.byref(st)), "tat_service_get_stats")
    return st.as_dict()


# learned primal-dual kernels (include/tat_lpd.h); pointers are ints, 0 for NULL

def tat_lpd_scratch_floats(batch, H, W) -> int:
    return int(load().tat_lpd_scratch_floats(batch, H, W))


def tat_conv_in_fwd(batch, H, W, cin, x0, x1, x2, w, b, h, stream=0):
    _check(load().tat_conv_in_fwd(batch, H, W, cin, x0, x1, x2 or None, w, b, h, stream or None), "tat_conv_in_fwd")


def tat_conv_in_bwd_data(batch, H, W, cin, g_h, h, w, gx0, gx1, gx2, accumulate, stream=0):
    _check(load().tat_conv_in_bwd_data(batch, H, W, cin, g_h, h or None, w, gx0 or None, gx1 or None, gx2 or None,
                                       accumulate, stream or None), "tat_conv_in_bwd_data")


def tat_conv_in_bwd_weights(batch, H, W, cin, x0, x1, x2, g_h, h, scratch, scratch_floats, gw, gb, stream=0):
    _check(load().tat_conv_in_bwd_weights(batch, H, W, cin, x0, x1, x2 or None, g_h, h or None, scratch, scratch_floats, gw,
                                          gb, stream or None), "tat_conv_in_bwd_weights")


def tat_conv_in_bwd(batch, H, W, cin, x0, x1, x2, g_h, h, w, gx0, gx1, gx2, accumulate, scratch, scratch_floats, gw,
                    gb, stream=0):
    _check(load().tat_conv_in_bwd(batch, H, W, cin, x0 or None, x1 or None, x2 or None, g_h, h or None, w or None,
                                  gx0 or None,
                                  gx1 or None, gx2 or None, accumulate, scratch or None, scratch_floats, gw or None,
                                  gb or None, stream or None), "tat_conv_in_bwd")


def tat_conv_mid_fwd(batch, H, W, h_in, w, b, h_out, stream=0):
    _check(load().tat_conv_mid_fwd(batch, H, W, h_in, w, b, h_out, stream or None), "tat_conv_mid_fwd")


def tat_conv_mid_bwd_data(batch, H, W, g_out, h_out, w, h_in, g_in, stream=0):
    _check(load().tat_conv_mid_bwd_data(batch, H, W, g_out, h_out or None, w, h_in or None, g_in, stream or None),
           "tat_conv_mid_bwd_data")


def tat_conv_mid_bwd_weights(batch, H, W, h_in, g_out, h_out, scratch, scratch_floats, gw, gb, stream=0):
    _check(load().tat_conv_mid_bwd_weights(batch, H, W, h_in, g_out, h_out or None, scratch, scratch_floats, gw, gb,
                                           stream or None), "tat_conv_mid_bwd_weights")


def tat_conv_out_fwd(batch, H, W, h, w, b, residual, out, stream=0):
    _check(load().tat_conv_out_fwd(batch, H, W, h, w, b, residual, out, stream or None), "tat_conv_out_fwd")


def tat_conv_out_bwd(batch, H, W, g_out, h, w, mask_relu, g_h, scratch, scratch_floats, gw, gb, stream=0):
    _check(load().tat_conv_out_bwd(batch, H, W, g_out, h, w, int(mask_relu), g_h, scratch, scratch_floats, gw, gb,
                                   stream or None), "tat_conv_out_bwd")


def tat_adam(count, lr, beta1, beta2, eps, step, param, grad, m, v, w_bf16, stream=0):
    _check(load().tat_adam(count, lr, beta1, beta2, eps, step, param, grad, m, v, w_bf16 or None, stream or None),
           "tat_adam")


def tat_lpd_timeout_probe(tries, gave_up_ptr, stream=0):
    _check(load().tat_lpd_timeout_probe(tries, gave_up_ptr, stream or None), "tat_lpd_timeout_probe")


def tat_lpd_check():
    """Raises TatError (timeout) if a tensor-core convolution gave up waiting for a TMA tile copy."""
    _check(load().tat_lpd_check(), "tat_lpd_check")


def tat_fill(count, value, out, stream=0):
    _check(load().tat_fill(count, value, out, stream or None), "tat_fill")


def tat_to_bf16(count, x, out, stream=0):
    _check(load().tat_to_bf16(count, x, out, stream or None), "tat_to_bf16")


def tat_mse(count, a, b, scale, grad, loss, stream=0):
    _check(load().tat_mse(count, a, b, scale, grad or None, loss, stream or None), "tat_mse")


def tat_status_string(status: int) -> str:
    return load().tat_status_string(status).decode()


def tat_debug_bessel(x: float, kmax: int):
    out = (_D * (kmax + 1))()
    _check(load().tat_debug_bessel(x, kmax, out), "tat_debug_bessel")
    return list(out)


def tat_debug_low_mode_rule():
    cnt = _I(0)
    _check(load().tat_debug_low_mode_rule(None, None, ctypes.byref(cnt)), "tat_debug_low_mode_rule")
    x, w = (_D * cnt.value)(), (_D * cnt.value)()
    _check(load().tat_debug_low_mode_rule(x, w, ctypes.byref(cnt)), "tat_debug_low_mode_rule")
    return list(x), list(w)


def tat_debug_stencils(desc: tat_plan_desc, rings, lps):
    m = len(rings)
    r = (_I * m)(*rings)
    l = (_I * m)(*lps)
    i0, k0, a, b = (_I * m)(), (_I * m)(), (_D * m)(), (_D * m)()
    _check(load().tat_debug_stencils(ctypes.byref(desc), r, l, i0, k0, a, b, m), "tat_debug_stencils")
    return list(i0), list(k0), list(a), list(b)


# ------------------------------------------------------------------ torch wrapper

class TatOperator:
    """A plan plus torch-managed workspace: ``forward(f)`` = A f, ``adjoint(g)`` = A* g.

    f: float32 CUDA tensor (n, n) or (B, n, n); g: (n_det, n_t) or (B, n_det, n_t).
    All arithmetic runs in libtat's kernels on the current torch stream.
    """

    def __init__(self, n, n_det, n_t, c=1.0, R=1.0, T=2.0, device=None, **desc_kw):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        desc = tat_plan_desc_default(n, n_det, n_t, c, R, T)
        for k, v in desc_kw.items():
            if k == "arc_len" and v is None:
                v = 2 * math.pi
            setattr(desc, k, v)
        self.desc = desc
        with torch.cuda.device(self.device):
            self.plan = tat_plan_create_ex(desc)
        self.info = tat_plan_get_info(self.plan)
        self.n, self.n_det, self.n_t = n, n_det, n_t
        # inner-product weights of X and Y (Eq. innerProducts): A* = W_X^{-1} A^T W_Y
        self.W_X = (self.info["h"] * R) ** 2
        self.W_Y = (self.info["dt"] * R / c) * (2 * math.pi * R / n_det)
        self._ws = {}

    def autotune(self, batch):
        """Times the column-strip, row-pair and column-CTA launch shapes on one A + A* of `batch`
        zero images and keeps the fastest for this plan (tat_plan_autotune); returns (ms, strip,
        row_pairs, cols_threads, row_threads)."""
        torch = self.torch
        f = torch.zeros((batch, self.n, self.n), dtype=torch.float32, device=self.device)
        g = torch.zeros((batch, self.n_det, self.n_t), dtype=torch.float32, device=self.device)
        ws = self.workspace(batch)
        with torch.cuda.device(self.device):
            return tat_plan_autotune(self.plan, batch, f.data_ptr(), g.data_ptr(), f.data_ptr(), ws.data_ptr(),
                                     torch.cuda.current_stream(self.device).cuda_stream)

    def workspace(self, batch):
        ws = self._ws.get(batch)
        if ws is None:
            nbytes = tat_workspace_size(self.plan, batch)
            ws = self.torch.empty(nbytes // 4 + 64, dtype=self.torch.float32, device=self.device)
            self._ws = {batch: ws}
        return ws

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def forward(self, f, out=None):
        torch = self.torch
        single = f.dim() == 2
        fb = f.reshape(-1, self.n, self.n)
        if fb.dtype != torch.float32 or not fb.is_cuda or not fb.is_contiguous():
            raise ValueError("f must be a contiguous float32 CUDA tensor")
        B = fb.shape[0]
        g = out if out is not None else torch.empty((B, self.n_det, self.n_t), dtype=torch.float32, device=fb.device)
        ws = self.workspace(B)
        with torch.cuda.device(self.device):
            tat_forward_batched(self.plan, B, fb.data_ptr(), self.n * self.n, g.data_ptr(), self.n_det * self.n_t,
                                ws.data_ptr(), self._stream())
        return g[0] if single and out is None else g

    def adjoint(self, g, out=None):
        torch = self.torch
        single = g.dim() == 2
        gb = g.reshape(-1, self.n_det, self.n_t)
        if gb.dtype != torch.float32 or not gb.is_cuda or not gb.is_contiguous():
            raise ValueError("g must be a contiguous float32 CUDA tensor")
        B = gb.shape[0]
        f = out if out is not None else torch.empty((B, self.n, self.n), dtype=torch.float32, device=gb.device)
        ws = self.workspace(B)
        with torch.cuda.device(self.device):
            tat_adjoint_batched(self.plan, B, gb.data_ptr(), self.n_det * self.n_t, f.data_ptr(), self.n * self.n,
                                ws.data_ptr(), self._stream())
        return f[0] if single and out is None else f

    def inverse(self, g, out=None):
        """f ~ A^{-1} g (Algorithm 3) for (n_det, n_t) or (B, n_det, n_t) data."""
        torch = self.torch
        single = g.dim() == 2
        gb = g.reshape(-1, self.n_det, self.n_t)
        if gb.dtype != torch.float32 or not gb.is_cuda or not gb.is_contiguous():
            raise ValueError("g must be a contiguous float32 CUDA tensor")
        B = gb.shape[0]
        f = out if out is not None else torch.empty((B, self.n, self.n), dtype=torch.float32, device=gb.device)
        ws = self.workspace(B)
        with torch.cuda.device(self.device):
            tat_inverse_batched(self.plan, B, gb.data_ptr(), self.n_det * self.n_t, f.data_ptr(), self.n * self.n,
                                ws.data_ptr(), self._stream())
        return f[0] if single and out is None else f

    def close(self):
        if getattr(self, "plan", None):
            tat_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TatService:
    """Mixed-size request runtime (include/tat_service.h) on the current CUDA device.

    ``submit(desc_kw, op, x, out)`` queues op(x) -> out for the problem described by
    ``desc_kw`` (n, n_det, n_t and optional tat_plan_desc fields); x and out are
    contiguous float32 CUDA tensors, or pinned host tensors (then the service uploads and
    downloads them on the request's slot stream); both must stay alive until ``synchronize``.
    """

    OPS = {"forward": TAT_OP_FORWARD, "adjoint": TAT_OP_ADJOINT, "inverse": TAT_OP_INVERSE, "pair": TAT_OP_PAIR}

    def __init__(self, memory_budget=None, max_batch=None, use_graphs=True, autotune=False, one_graph=True):
        cfg = tat_service_config_default()
        if memory_budget is not None:
            cfg.memory_budget = int(memory_budget)
        if max_batch is not None:
            cfg.max_batch = int(max_batch)
        cfg.use_graphs = 1 if use_graphs else 0
        cfg.autotune = 1 if autotune else 0
        cfg.one_graph = 1 if one_graph else 0
        self.handle = tat_service_create(cfg)
        self._keep = []

    @staticmethod
    def desc(n, n_det, n_t, c=1.0, R=1.0, T=2.0, **kw):
        d = tat_plan_desc_default(n, n_det, n_t, c, R, T)
        for k, v in kw.items():
            setattr(d, k, v)
        return d

    def submit(self, desc, op, x, out):
        for t in (x, out):
            if not ((t.is_cuda or t.is_pinned()) and t.is_contiguous() and t.dtype.itemsize == 4):
                raise ValueError("x and out must be contiguous float32 CUDA or pinned host tensors")
        self._keep.append((x, out))
        return tat_service_submit(self.handle, desc, self.OPS[op], x.data_ptr(), out.data_ptr())

    def flush(self):
        tat_service_flush(self.handle)

    def synchronize(self):
        tat_service_synchronize(self.handle)
        self._keep = []

    def latency(self, rid):
        return tat_service_latency(self.handle, rid)

    def stats(self):
        return tat_service_get_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            tat_service_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
