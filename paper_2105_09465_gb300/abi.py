"""ctypes binding of liblensgp.so (the C ABI in include/lensgp.h).

Argument marshalling only: every computation runs in the CUDA library. Tensors
cross the boundary as raw device pointers, the stream as the current torch
CUDA stream's handle. Loading fails loudly when the library is missing; there
is no fallback.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

from .build import LIB_PATH, build

LR_OK = 0
LR_ERR_INVALID_ARG = 1
LR_ERR_CUDA = 2
LR_ERR_OUT_OF_MEMORY = 3
LR_ERR_TIMEOUT = 4
LR_PENDING = 5
LR_ERR_NOT_FOUND = 6
LR_ERR_BUSY = 7

LR_PROFILE_TNFW = 0
LR_PROFILE_POINT_MASS = 1


class LensGPError(RuntimeError):
    def __init__(self, status: int, func: str, msg: str):
        super().__init__(f"{func} failed with status {status}: {msg}")
        self.status = status


class lr_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("ss", ctypes.c_int32),
                ("pix", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


class lr_lens(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("x0", "y0", "q", "phi", "theta_e", "gamma", "g1", "g2")]


class lr_points(ctypes.Structure):
    _fields_ = [("xy", ctypes.c_void_p), ("grid", lr_grid), ("n", ctypes.c_int64),
                ("lens", ctypes.POINTER(lr_lens)), ("sub", ctypes.c_void_p), ("n_sub", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("lens_record", ctypes.c_void_p)]


class lr_grads(ctypes.Structure):
    _fields_ = [("d_v", ctypes.c_void_p), ("d_x", ctypes.c_void_p), ("d_y", ctypes.c_void_p),
                ("d_lengthscale", ctypes.c_void_p), ("d_variance", ctypes.c_void_p), ("d_lens", ctypes.c_void_p),
                ("d_sub", ctypes.c_void_p), ("beta_in", ctypes.c_void_p),
                ("moments_in", ctypes.c_void_p), ("source_rows", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("row0", ctypes.c_int64)]


class lr_session_cfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int32), ("device", ctypes.c_int32),
                ("fill_pairs", ctypes.c_int64)]


class lr_request(ctypes.Structure):
    _fields_ = [("grid", lr_grid), ("lens", lr_lens), ("sub", ctypes.c_void_p), ("n_sub", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("ygrid", lr_grid), ("v0", ctypes.c_void_p), ("data", ctypes.c_void_p),
                ("lengthscale", ctypes.c_float), ("variance", ctypes.c_float), ("step", ctypes.c_float),
                ("iters", ctypes.c_int32)]


class lr_result(ctypes.Structure):
    _fields_ = [("out", ctypes.c_void_p), ("v", ctypes.c_void_p), ("d_lens", ctypes.c_void_p),
                ("d_sub", ctypes.c_void_p), ("d_lengthscale", ctypes.c_double), ("d_variance", ctypes.c_double),
                ("loss", ctypes.c_double), ("t_submit_s", ctypes.c_double), ("t_admit_s", ctypes.c_double),
                ("t_done_s", ctypes.c_double)]


class lr_session_stats(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_int64), ("active", ctypes.c_int64), ("held", ctypes.c_int64),
                ("used_bytes", ctypes.c_size_t), ("iterations", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("active_pairs", ctypes.c_int64), ("peak_active_pairs", ctypes.c_int64)]


_P = ctypes.c_void_p
_lib = None

# name -> (restype, argtypes); every symbol include/lensgp.h declares
SIGNATURES = {
    "lr_last_error": (ctypes.c_char_p, []),
    "lr_status_name": (ctypes.c_char_p, [ctypes.c_int32]),
    "lr_probe_pipe_rates": (ctypes.c_int32, [ctypes.c_int32, _P, _P, _P, _P]),
    "lr_fault_status": (ctypes.c_int32, [_P, ctypes.c_int32]),
    "lr_selftest_bounded_wait": (ctypes.c_int32, [ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]),
    "lr_kernel_timer_enable": (ctypes.c_int32, [ctypes.c_int32]),
    "lr_kernel_timer_read": (ctypes.c_int32, [ctypes.c_int32, _P, _P, _P]),
    "lr_set_pair_culling": (ctypes.c_int32, [ctypes.c_int32]),
    "lr_cull_pairs_evaluated": (ctypes.c_int32, [ctypes.POINTER(lr_points), ctypes.POINTER(lr_points), ctypes.c_float,
                                                 ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                                 ctypes.POINTER(ctypes.c_int64), _P]),
    "lens_raytrace": (ctypes.c_int32, [ctypes.POINTER(lr_points), _P, _P, _P]),
    "lr_grid_points": (ctypes.c_int32, [ctypes.POINTER(lr_grid), _P, _P]),
    "lr_lens_record_bytes": (ctypes.c_size_t, []),
    "lr_lens_prepare": (ctypes.c_int32, [_P, ctypes.c_float, _P, _P]),
    "lr_vec_axpby": (ctypes.c_int32, [ctypes.c_int64, ctypes.c_float, _P, ctypes.c_float, _P, _P, _P]),
    "lr_vec_mul": (ctypes.c_int32, [ctypes.c_int64, _P, _P, _P, _P]),
    "lr_vec_pack": (ctypes.c_int32, [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P]),
    "lr_sum_scalars": (ctypes.c_int32, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32, _P, _P]),
    "lens_jacobian": (ctypes.c_int32, [ctypes.POINTER(lr_points), _P, _P, _P]),
    "gp_kernel_matvec": (ctypes.c_int32, [ctypes.POINTER(lr_points), ctypes.POINTER(lr_points), _P, ctypes.c_int32,
                                          ctypes.c_float, ctypes.c_float, _P, _P, _P, ctypes.c_size_t, _P]),
    "lr_matvec_workspace_size": (ctypes.c_int32, [ctypes.POINTER(lr_points), ctypes.POINTER(lr_points),
                                                  ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "gp_kernel_matvec_static_scratch": (ctypes.c_int32, [ctypes.POINTER(lr_points), ctypes.POINTER(lr_points), _P,
                                                         ctypes.c_int32, ctypes.c_float, ctypes.c_float, _P, _P,
                                                         _P]),
    "lr_static_scratch_bytes": (ctypes.c_size_t, []),
    "gp_pixel_shapes": (ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P]),
    "gp_windowed_matvec": (ctypes.c_int32, [_P, _P, ctypes.c_int64, ctypes.POINTER(lr_grid), ctypes.POINTER(lr_points),
                                            _P, ctypes.c_float, _P, _P, ctypes.c_size_t, _P]),
    "gp_knn_density": (ctypes.c_int32, [_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, _P, _P, _P,
                                        ctypes.c_size_t, _P]),
    "lr_knn_workspace_size": (ctypes.c_int32, [ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]),
    "gp_kernel_matvec_train": (ctypes.c_int32, [ctypes.POINTER(lr_points), ctypes.POINTER(lr_points), _P,
                                                ctypes.c_int32, ctypes.c_float, ctypes.c_float, _P, _P, _P, _P,
                                                ctypes.c_size_t, _P]),
    "lr_matvec_train_workspace_size": (ctypes.c_int32, [ctypes.POINTER(lr_points), ctypes.POINTER(lr_points),
                                                        ctypes.c_int32, ctypes.POINTER(ctypes.c_size_t)]),
    "lr_grid_pairs_evaluated": (ctypes.c_int32, [_P, ctypes.c_int64, ctypes.POINTER(lr_grid), ctypes.POINTER(lr_grid),
                                                 ctypes.c_float, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), _P]),
    "lr_elbo_workspace_size": (ctypes.c_size_t, []),
    "gp_gaussian_nll": (ctypes.c_int32, [_P, ctypes.c_int64, ctypes.POINTER(lr_grid), _P, _P, ctypes.c_float, _P, _P,
                                         _P, _P, ctypes.c_size_t, _P]),
    "gp_diag_normal_draw": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int64, ctypes.c_float, _P, _P, _P, ctypes.c_size_t,
                                             _P]),
    "gp_diag_normal_vjp": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int64, ctypes.c_float, _P, ctypes.c_double,
                                            ctypes.c_double, _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "gp_partial_mvn_draw": (ctypes.c_int32, [_P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_int64, _P, _P, _P,
                                             ctypes.c_size_t, _P]),
    "gp_partial_mvn_vjp": (ctypes.c_int32, [_P, _P, _P, ctypes.c_int32, ctypes.c_int64, _P, ctypes.c_double, _P, _P,
                                            _P, _P, _P]),
    "gp_windowed_matvec_bwd": (ctypes.c_int32, [_P, _P, ctypes.c_int64, ctypes.POINTER(lr_grid),
                                                ctypes.POINTER(lr_points), _P, ctypes.c_float, _P, _P, _P, _P, _P, _P,
                                                _P, ctypes.c_size_t, _P]),
    "lr_windowed_bwd_workspace_size": (ctypes.c_int32, [ctypes.c_int64, ctypes.POINTER(lr_grid),
                                                        ctypes.POINTER(lr_points), ctypes.POINTER(ctypes.c_size_t)]),
    "lr_windowed_pairs_evaluated": (ctypes.c_int32, [_P, _P, ctypes.c_int64, ctypes.POINTER(lr_grid),
                                                     ctypes.POINTER(lr_points), ctypes.c_float, ctypes.c_int32,
                                                     ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                                     _P]),
    "gp_pixel_shapes_vjp": (ctypes.c_int32, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "gp_windowed_matvec_nll": (ctypes.c_int32, [_P, _P, ctypes.c_int64, ctypes.POINTER(lr_grid),
                                                ctypes.POINTER(lr_points), _P, ctypes.c_float, _P, _P, ctypes.c_float,
                                                _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "lr_windowed_workspace_size": (ctypes.c_int32, [ctypes.c_int64, ctypes.POINTER(lr_grid),
                                                    ctypes.POINTER(lr_points), ctypes.POINTER(ctypes.c_size_t)]),
    "gp_kernel_matvec_layers": (ctypes.c_int32, [ctypes.POINTER(lr_points), ctypes.POINTER(lr_points), ctypes.c_int32,
                                                 _P, _P, _P, ctypes.c_int32, _P, _P, _P, ctypes.c_size_t, _P]),
    "lr_matvec_layers_workspace_size": (ctypes.c_int32, [ctypes.POINTER(lr_points), ctypes.POINTER(lr_points),
                                                         ctypes.c_int32, ctypes.c_int32,
                                                         ctypes.POINTER(ctypes.c_size_t)]),
    "gp_kernel_matvec_bwd": (ctypes.c_int32, [ctypes.POINTER(lr_points), ctypes.POINTER(lr_points), _P,
                                              ctypes.c_int32, ctypes.c_float, ctypes.c_float, _P,
                                              ctypes.POINTER(lr_grads), _P, ctypes.c_size_t, _P]),
    "lr_matvec_bwd_workspace_size": (ctypes.c_int32, [ctypes.POINTER(lr_points), ctypes.POINTER(lr_points),
                                                      ctypes.c_int32, ctypes.POINTER(lr_grads),
                                                      ctypes.POINTER(ctypes.c_size_t)]),
    "lens_raytrace_vjp": (ctypes.c_int32, [ctypes.POINTER(lr_points), _P, _P, _P, _P, ctypes.c_size_t, _P]),
    "lr_raytrace_vjp_workspace_size": (ctypes.c_int32, [ctypes.POINTER(lr_points), ctypes.POINTER(ctypes.c_size_t)]),
    "solve_session_create": (ctypes.c_int32, [ctypes.POINTER(lr_session_cfg), ctypes.POINTER(ctypes.c_void_p)]),
    "solve_session_submit": (ctypes.c_int32, [_P, ctypes.POINTER(lr_request), ctypes.POINTER(ctypes.c_uint64)]),
    "solve_session_poll": (ctypes.c_int32, [_P, ctypes.c_uint64, ctypes.POINTER(lr_result), ctypes.c_int64]),
    "solve_session_cancel": (ctypes.c_int32, [_P, ctypes.c_uint64]),
    "solve_session_inject_fault": (ctypes.c_int32, [_P]),
    "solve_session_stats": (ctypes.c_int32, [_P, ctypes.POINTER(lr_session_stats)]),
    "solve_session_destroy": (ctypes.c_int32, [_P]),
}


def load(path: str | Path | None = None, build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads (building first if needed) liblensgp.so and declares every entry point."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        if not build_if_missing:
            raise FileNotFoundError(f"{p} is missing: build it with paper_2105_09465_gb300.build.build()")
        build()
    lib = ctypes.CDLL(str(p))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(status: int, func: str) -> None:
    if status != LR_OK:
        msg = load().lr_last_error().decode(errors="replace")
        raise LensGPError(status, func, msg)
