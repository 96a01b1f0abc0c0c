"""ctypes declarations of the C ABI in include/ica.h (loads libica.so; no fallback)."""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libica.so")

# ica_status codes (include/ica.h)
ICA_OK = 0
ICA_ERR_ARG = 1
ICA_ERR_CUDA = 2
ICA_ERR_NONFINITE = 3
ICA_ERR_ILLCOND = 4
ICA_ERR_TIMEOUT = 5
ICA_ERR_WORKSPACE = 6
ICA_ERR_UNSUPPORTED = 7

# ica_precision
ICA_FP32 = 0
ICA_BF16 = 1
ICA_FP8 = 2
ICA_PLAIN_FP32 = 3


class ica_opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("gauss_test", C.c_int),
        ("refine_topk", C.c_int),
        ("refine_iters", C.c_int),
        ("stage_tol", C.c_double),
        ("refine_tol", C.c_double),
        ("fp32_tol_floor", C.c_double),
        ("B0", C.c_void_p),
        ("max_splits", C.c_int),
        ("profile", C.c_int),
        ("prune_params", C.c_void_p),
        ("prune_tau", C.c_float),
        ("record_features", C.c_void_p),
        ("record_labels", C.c_void_p),
        ("stage_persistent", C.c_int),
        ("wait_ns", C.c_int64),
        ("stall_test", C.c_int),
        ("prune_keep_frac", C.c_float),
        ("prune_cos", C.c_float),
        ("prune_gauss", C.c_int),
        ("algorithm", C.c_int),
        ("stage_lo_from", C.c_int),
        ("stage_streamk", C.c_int),
        ("record_cands", C.c_void_p),
        ("fp8_iters", C.c_int),
    ]


class ica_dataset(C.Structure):
    _fields_ = [
        ("Xw", C.c_void_p),
        ("N", C.c_int),
        ("T", C.c_int64),
        ("n_components", C.c_int),
        ("W_out", C.c_void_p),
        ("kurt_out", C.c_void_p),
        ("n_found", C.POINTER(C.c_int)),
    ]


# learned restart pruner (include/ica.h)
ICA_MLP_IN = 13
ICA_MLP_HIDDEN = 64
ICA_MLP_PARAMS = 5147


vp, i32, i64, u64, f64, sz, f32 = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double, C.c_size_t, C.c_float

# name -> (restype, argtypes); exactly the functions declared in include/ica.h
SIGNATURES = {
    "ica_default_opts": (None, [C.POINTER(ica_opts)]),
    "ica_status_string": (C.c_char_p, [i32]),
    "ica_last_error": (C.c_char_p, []),
    "ica_create": (i32, [C.POINTER(vp), i32]),
    "ica_destroy": (i32, [vp]),
    "ica_set_stream": (i32, [vp, vp]),
    "ica_workspace_bytes": (sz, [i32, i64, i32, C.POINTER(ica_opts)]),
    "ica_set_workspace": (i32, [vp, vp, sz]),
    "ica_whiten": (i32, [vp, vp, i32, i64, vp, vp, vp]),
    "ica_order_fit": (i32, [vp, vp, i32, i64, i32, i32, i32, f64, u64, C.POINTER(ica_opts), vp, vp, C.POINTER(i32)]),
    "ica_last_stats": (i32, [vp, C.c_char_p, sz]),
    "ica_init_restarts": (i32, [vp, u64, i32, i32, i32, vp, i32]),
    "ica_deflation_basis": (i32, [vp, vp, i32, i32, vp]),
    "ica_reduce": (i32, [vp, vp, i32, i32, vp, i64, vp, i64, vp, i64]),
    "ica_quantize_e4m3": (i32, [vp, vp, i32, i64, i64, vp, i64, vp]),
    "ica_fp_step": (i32, [vp, i32, vp, i32, i32, vp, i64, i64, vp, vp]),
    "ica_kurtosis": (i32, [vp, i32, vp, i32, i32, vp, i64, i64, vp, vp]),
    "ica_fp_step_noalloc": (i32, [i32, vp, i32, i32, vp, i64, i64, vp, vp, vp]),
    "ica_batched_workspace_bytes": (sz, [C.POINTER(ica_dataset), i32, i32, C.POINTER(ica_opts), i32]),
    "ica_order_fit_batched": (i32, [vp, C.POINTER(ica_dataset), i32, i32, i32, f64, u64, C.POINTER(ica_opts), i32]),
    "ica_mlp_init": (i32, [vp, u64, vp]),
    "ica_mlp_standardize": (i32, [vp, vp, i32, vp]),
    "ica_mlp_forward": (i32, [vp, vp, vp, i32, i32, vp]),
    "ica_mlp_scratch_bytes": (sz, [i32]),
    "ica_mlp_train_step": (i32, [vp, vp, vp, vp, i32, vp, vp, i32, f32, f32, i32, vp, sz, vp, vp]),
}

_lib = None


def load() -> C.CDLL:
    """Load libica.so (raises if it has not been built: there is no other implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
