"""ctypes declarations of the C ABI in include/gpf.h and the loader of
libgpf.so. Loading fails loudly when the library is missing: there is no
fallback implementation."""

from __future__ import annotations

import ctypes
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgpf.so")

GPF_OK = 0
GPF_ERR_INVALID_ARG = 1
GPF_ERR_CUDA = 2
GPF_ERR_WORKSPACE_TOO_SMALL = 3
GPF_ERR_CAPACITY = 4
GPF_ERR_NOT_BUILT = 5
GPF_ERR_MISMATCH = 6
GPF_ERR_TIMEOUT = 7
GPF_ERR_NONFINITE = 8
GPF_FLAG_CAPACITY = 1
GPF_FLAG_TIMEOUT = 2
GPF_FLAG_NONFINITE = 4
GPF_BWD_SPLIT_WAYS = 16
GPF_BWD_SPLIT_MAX = 16384
GPF_PEAK_FP32_FMA = 0
GPF_PEAK_EX2 = 1

GPF_SUM = 0
GPF_NORMALIZED = 1
GPF_DISK_KDE = 2
GPF_MAX_CHANNELS = 8
GPF_MAX_DIM = 1024
GPF_MAX_LEVELS = 16
GPF_MAX_COOP_CELLS = 8
GPF_F32 = 0
GPF_BF16 = 1
GPF_BF16_MEAN32 = 2
GPF_BF16_GROUP = 16
GPF_NB_KSIGMA = 0
GPF_NB_BALL_KNN = 1
GPF_MAX_KMIN = 16

c_i32, c_i64, c_f32, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p


class gpf_field(ctypes.Structure):
    _fields_ = [("n", c_i64), ("channels", c_i32), ("storage", c_i32), ("mean", c_vp),
                ("quat", c_vp), ("logscale", c_vp), ("spectrum", c_vp), ("anchor", c_vp)]


class gpf_queries(ctypes.Structure):
    _fields_ = [("m", c_i64), ("x", c_vp), ("normal", c_vp), ("wo", c_vp), ("albedo", c_vp),
                ("valid", c_vp)]


class gpf_query_params(ctypes.Structure):
    _fields_ = [("mode", c_i32), ("r_max", c_f32), ("eps", c_f32), ("neighbourhood", c_i32),
                ("ball_r", c_f32), ("k_min", c_i32), ("f64_sums", c_i32)]


class gpf_grid_config(ctypes.Structure):
    _fields_ = [("origin", c_f32 * 3), ("cell_size", c_f32), ("levels", c_i32),
                ("max_span", c_i32), ("query_level", c_i32), ("dims", c_i32 * 3),
                ("hash_bits", c_i32), ("channels", c_i32), ("cutoff_sigma", c_f32), ("brute_force", c_i32),
                ("coop_cells", c_i32), ("field_storage", c_i32), ("ball_radius", c_f32),
                ("max_gaussians", c_i64), ("max_queries", c_i64), ("max_pairs", c_i64),
                ("max_nb_pairs", c_i64), ("split_items", c_i32), ("tile_order", c_i32)]


class gpf_index_stats_t(ctypes.Structure):
    _fields_ = [("n_pairs", c_i64), ("n_active", c_i64), ("n_live", c_i64), ("n_small", c_i64),
                ("n_huge", c_i64), ("n_split", c_i64), ("level_mask", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("overflow", c_i32), ("n_hybrid_units", c_i32),
                ("n_nb_pairs", c_i64)]


class gpf_field_grad(ctypes.Structure):
    _fields_ = [("mean", c_vp), ("quat", c_vp), ("logscale", c_vp), ("spectrum", c_vp),
                ("accumulate", c_i32), ("reserved", c_i32)]


class gpf_adam_hparams(ctypes.Structure):
    _fields_ = [("lr", c_f32 * 4), ("beta1", c_f32), ("beta2", c_f32), ("eps", c_f32),
                ("step", c_i32), ("step_counter", c_vp), ("guard", c_vp)]


# name -> (restype, argtypes); every symbol include/gpf.h declares
SIGNATURES = {
    "gpf_version": (ctypes.c_char_p, []),
    "gpf_status_string": (ctypes.c_char_p, [c_i32]),
    "gpf_last_error": (ctypes.c_char_p, []),
    "gpf_index_create": (c_i32, [ctypes.POINTER(gpf_grid_config), ctypes.POINTER(c_vp)]),
    "gpf_index_destroy": (None, [c_vp]),
    "gpf_index_workspace_size": (c_i32, [c_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "gpf_build_index": (c_i32, [c_vp, ctypes.POINTER(gpf_field), ctypes.POINTER(gpf_queries),
                                c_vp, ctypes.c_size_t, c_vp]),
    "gpf_index_stats": (c_i32, [c_vp, ctypes.POINTER(gpf_index_stats_t), c_vp]),
    "gpf_index_flags_async": (c_i32, [c_vp, c_vp, c_vp]),
    "gpf_radiance_fwd": (c_i32, [c_vp, ctypes.POINTER(gpf_field), ctypes.POINTER(gpf_queries),
                                 ctypes.POINTER(gpf_query_params), c_vp, c_vp, c_vp]),
    "gpf_count_pairs": (c_i32, [c_vp, ctypes.POINTER(gpf_field), ctypes.POINTER(gpf_queries),
                                c_vp, c_vp]),
    "gpf_launch_count": (ctypes.c_uint64, []),
    "gpf_field_quantize": (c_i32, [ctypes.POINTER(gpf_field), ctypes.POINTER(gpf_field), c_vp]),
    "gpf_index_set_timing_events": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "gpf_radiance_bwd": (c_i32, [c_vp, ctypes.POINTER(gpf_field), ctypes.POINTER(gpf_queries),
                                 ctypes.POINTER(gpf_query_params), c_vp, c_vp, c_vp,
                                 ctypes.POINTER(gpf_field_grad), c_vp]),
    "gpf_mse_workspace_size": (c_i32, [c_i64, ctypes.POINTER(ctypes.c_size_t)]),
    "gpf_mse_loss_grad": (c_i32, [c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                  ctypes.c_size_t, c_vp]),
    "gpf_mse_loss_grad_noalloc": (c_i32, [c_i64, c_i32, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "gpf_adam_step": (c_i32, [ctypes.POINTER(gpf_field), ctypes.POINTER(gpf_field_grad),
                              ctypes.POINTER(gpf_field_grad), ctypes.POINTER(gpf_field_grad),
                              ctypes.POINTER(gpf_adam_hparams), c_vp]),
    "gpf_sort_pairs_workspace_size": (c_i32, [c_i64, ctypes.POINTER(ctypes.c_size_t)]),
    "gpf_sort_pairs": (c_i32, [c_vp, c_vp, c_vp, c_vp, c_i64, c_i32, c_vp, ctypes.c_size_t,
                               ctypes.POINTER(c_i32), c_vp]),
    "gpf_sort_pairs_check": (c_i32, [c_vp, c_vp]),
    "gpf_test_sort_wait_timeout": (c_i32, [ctypes.c_uint32, c_vp]),
    "gpf_measure_alu_peak": (c_i32, [c_i32, c_i32, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


class GPFError(RuntimeError):
    """A libgpf call returned a status other than GPF_OK."""

    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


def load() -> ctypes.CDLL:
    """Load libgpf.so once. Raises when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libgpf.so not found at {LIB_PATH}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, what: str) -> None:
    if status != GPF_OK:
        lib = load()
        name = lib.gpf_status_string(status).decode()
        msg = lib.gpf_last_error().decode()
        raise GPFError(status, f"{what}: {name}: {msg}")
