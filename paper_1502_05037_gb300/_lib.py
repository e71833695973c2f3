"""ctypes binding of libpurify.so (the C ABI declared in include/purify.h).

Argument marshalling only: every step of the imaging path runs in the CUDA
library. Array arguments may be torch tensors (device or host) or NumPy
arrays (host); they are passed as raw pointers. Loading fails loudly when the
library has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpurify.so")

PURIFY_OK, PURIFY_EINVAL, PURIFY_ENOMEM, PURIFY_ECUDA, PURIFY_ETIMEOUT, PURIFY_ENOTCONV, PURIFY_ENAN = range(7)
PURIFY_F32, PURIFY_F64 = 0, 1
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOTCONV", 6: "ENAN"}


class purify_plan_desc(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("M", C.c_int64),
        ("u", C.c_void_p), ("v", C.c_void_p),
        ("R", C.c_int32),
        ("block_offsets", C.POINTER(C.c_int64)),
        ("kb_width", C.c_int32),
        ("oversample", C.c_double),
        ("kb_beta", C.c_double),
        ("levels", C.c_int32),
        ("basis_mask", C.c_uint32),
        ("dtype", C.c_int32),
        ("stream", C.c_void_p),
        ("tile", C.c_int32),
        ("grid_mode", C.c_int32),
    ]


class purify_plan_info(C.Structure):
    _fields_ = [
        ("Kx", C.c_int32), ("Ky", C.c_int32), ("q", C.c_int32), ("tile", C.c_int32),
        ("N", C.c_int64), ("D", C.c_int64), ("M", C.c_int64),
        ("R", C.c_int32), ("J", C.c_int32), ("levels", C.c_int32),
        ("beta", C.c_double),
        ("workspace_bytes", C.c_int64),
        ("grid_mode", C.c_int32),
        ("degrid_mode", C.c_int32),
        ("normal_mode", C.c_int32),
        ("lane_tile", C.c_int32),
        ("fft_rows_per_block", C.c_int32),
        ("fft_cols_per_block", C.c_int32),
        ("fft_cols_per_thread", C.c_int32),
    ]


class purify_sdmm_params(C.Structure):
    _fields_ = [
        ("max_iter", C.c_int32),
        ("cg_iters", C.c_int32),
        ("cg_tol", C.c_double),
        ("gamma", C.c_double),
        ("nu", C.c_double),
        ("rel_obj_tol", C.c_double),
        ("eps_tol", C.c_double),
        ("check_every", C.c_int32),
        ("resume", C.c_int32),
        ("toeplitz", C.c_int32),
        ("block_groups", C.c_int32),
        ("group_seq", C.POINTER(C.c_int32)),
    ]


class purify_pd_params(C.Structure):
    _fields_ = [
        ("iters", C.c_int32),
        ("tau", C.c_double),
        ("sigma", C.c_double),
        ("nu", C.c_double),
    ]


class purify_sdmm_stats(C.Structure):
    _fields_ = [
        ("iters", C.c_int32),
        ("cg_iters_total", C.c_int32),
        ("objective", C.c_double),
        ("max_resid_over_eps", C.c_double),
        ("rel_change", C.c_double),
        ("gamma", C.c_double),
        ("nu", C.c_double),
        ("status", C.c_int32),
    ]


class purify_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double)]


_P = C.c_void_p
_SIGS = {
    "purify_plan_create": (C.c_int, [C.POINTER(purify_plan_desc), C.POINTER(_P)]),
    "purify_plan_destroy": (C.c_int, [_P]),
    "purify_plan_set_stream": (C.c_int, [_P, _P]),
    "purify_plan_get_info": (C.c_int, [_P, C.POINTER(purify_plan_info)]),
    "purify_phi": (C.c_int, [_P, _P, _P]),
    "purify_phi_adj": (C.c_int, [_P, _P, _P]),
    "purify_phi_normal": (C.c_int, [_P, _P, _P]),
    "purify_fft2": (C.c_int, [_P, _P, C.c_int32]),
    "purify_psi": (C.c_int, [_P, _P, _P]),
    "purify_psi_adj": (C.c_int, [_P, _P, _P]),
    "purify_op_norm_sq": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_double)]),
    "purify_sdmm_solve": (C.c_int, [_P, _P, C.POINTER(C.c_double), _P, _P,
                                    C.POINTER(purify_sdmm_params), C.POINTER(purify_sdmm_stats)]),
    "purify_sdmm_iterate": (C.c_int, [_P, C.c_int32]),
    "purify_sdmm_iterate_groups": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int32)]),
    "purify_shard_iterate_local": (C.c_int, [_P, _P]),
    "purify_shard_cg_begin": (C.c_int, [_P, _P]),
    "purify_shard_cg_apply": (C.c_int, [_P, C.c_int32, _P]),
    "purify_shard_cg_combine": (C.c_int, [_P, C.c_int32, _P]),
    "purify_shard_iterate_end": (C.c_int, [_P, C.c_int32]),
    "purify_pd_solve": (C.c_int, [_P, _P, C.POINTER(C.c_double), _P, _P,
                                  C.POINTER(purify_pd_params), C.POINTER(purify_sdmm_stats)]),
    "purify_batch_create": (C.c_int, [C.POINTER(_P), C.c_int32, _P, C.POINTER(_P)]),
    "purify_batch_iterate": (C.c_int, [_P, C.c_int32]),
    "purify_batch_destroy": (C.c_int, [_P]),
    "purify_reweight": (C.c_int, [_P, _P, C.c_double, _P]),
    "purify_coef_std": (C.c_int, [_P, _P, C.POINTER(C.c_double)]),
    "purify_noise_sigma": (C.c_int, [C.c_double, C.c_int64, C.c_double, C.POINTER(C.c_double)]),
    "purify_chi2_epsilon": (C.c_int, [C.c_double, C.POINTER(C.c_int64), C.c_int32, C.POINTER(C.c_double)]),
    "purify_psi_adj_static": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_uint32, C.c_int32, _P]),
    "purify_conv2d": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P, _P, C.c_int32, C.c_int32,
                                C.c_int32, _P, _P]),
    "purify_unet_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_uint64, _P,
                                     C.POINTER(_P)]),
    "purify_unet_destroy": (C.c_int, [_P]),
    "purify_unet_num_params": (C.c_int64, [_P]),
    "purify_unet_get_params": (C.c_int, [_P, _P]),
    "purify_unet_set_params": (C.c_int, [_P, _P]),
    "purify_unet_forward": (C.c_int, [_P, _P, _P, C.c_int32]),
    "purify_unet_gradients": (C.c_int, [_P, _P, _P, C.c_int32, _P, C.POINTER(C.c_double)]),
    "purify_unet_train_step": (C.c_int, [_P, _P, _P, C.c_int32, C.c_float, C.POINTER(C.c_double)]),
    "purify_timing_enable": (C.c_int, [_P, C.c_int32]),
    "purify_timing_read": (C.c_int32, [_P, C.POINTER(purify_kernel_time), C.c_int32, C.c_int32]),
    "purify_launch_count": (C.c_int64, []),
    "purify_last_error": (C.c_char_p, []),
}

_lib = None


def load(path: str | None = None):
    """Load libpurify.so (once). Raises OSError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"libpurify.so not built ({path}); run paper_1502_05037_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


class PurifyError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int):
    if status != PURIFY_OK:
        raise PurifyError(status, load().purify_last_error().decode())
