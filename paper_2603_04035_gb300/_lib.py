"""ctypes declarations of libdrgb.so (the C ABI in include/drgb.h).

Loading fails loudly when the library has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdrgb.so")

OK = 0
ERR_INVALID = -1
ERR_WORKSPACE = -2
ERR_CUDA = -3
ERR_TIMEOUT = -4
ERR_NONFINITE = -5
ERR_DEVICE = -6
MAX_K = 32
STATIC_SCRATCH_BYTES = 16 << 20
TUNE_EPOCH_WARPS = 1
TUNE_EPOCH_PIPE = 2
FLAG_AUTOTUNE = 1
FLAG_INIT_SPECTRAL = 2

ERROR_NAMES = {ERR_INVALID: "invalid argument", ERR_WORKSPACE: "workspace too small",
               ERR_CUDA: "CUDA error", ERR_TIMEOUT: "device timeout",
               ERR_NONFINITE: "non-finite input", ERR_DEVICE: "unsupported device"}


class Params(C.Structure):
    _fields_ = [("k", C.c_int32), ("n_epochs", C.c_int32), ("neg", C.c_int32),
                ("lr0", C.c_float), ("min_dist", C.c_float), ("spread", C.c_float),
                ("init_range", C.c_float), ("seed_init", C.c_uint64), ("seed_neg", C.c_uint64),
                ("knn_mode", C.c_int32), ("flags", C.c_int32), ("pca_dim", C.c_int32)]


class MlpParams(C.Structure):
    _fields_ = [("steps", C.c_int32), ("batch_edges", C.c_int32), ("neg", C.c_int32), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64)]


EPOCH_CB = C.CFUNCTYPE(C.c_int, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p)

vp, i32, i64, u64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_float

SIGNATURES = {
    "drgb_version": (C.c_int, []),
    "drgb_ctx_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "drgb_ctx_destroy": (C.c_int, [vp]),
    "drgb_last_error": (C.c_char_p, [vp]),
    "drgb_sync": (C.c_int, [vp, vp]),
    "drgb_ctx_scratch_bytes": (C.c_int64, [vp]),
    "drgb_launch_count": (C.c_int64, [vp]),
    "drgb_set_tuning": (C.c_int, [vp, i32, i32]),
    "drgb_get_tuning": (C.c_int, [vp, i32, C.POINTER(i32)]),
    "drgb_set_tuning_cache": (C.c_int, [vp, C.c_char_p]),
    "drgb_tuning_cache_lookup": (C.c_int, [C.c_char_p, C.c_char_p, C.POINTER(i32), C.POINTER(i32)]),
    "drgb_tuning_cache_store": (C.c_int, [C.c_char_p, C.c_char_p, i32, i32]),
    "drgb_set_profiling": (C.c_int, [vp, C.c_int]),
    "drgb_stage_times": (C.c_int, [vp, C.POINTER(C.c_float), C.c_int]),
    "drgb_knn_graph": (C.c_int, [vp, vp, i64, i32, i32, i32, vp, vp, vp]),
    "drgb_knn_uncertified": (C.c_int, [vp, C.POINTER(C.c_int64), vp]),
    "drgb_knn_tiles": (C.c_int, [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), vp]),
    "drgb_set_scratch_limit": (C.c_int, [vp, i64]),
    "drgb_gather_probe": (C.c_int, [vp, vp, i64, i32, C.c_uint32, C.POINTER(C.c_double), vp]),
    "drgb_knn_nndescent": (C.c_int, [vp, vp, i64, i32, i32, u64, C.c_double, i32, i32, vp, vp,
                                     C.POINTER(C.c_int32), C.POINTER(C.c_double), vp]),
    "drgb_fuzzy_weights": (C.c_int, [vp, vp, vp, i64, i32, i32, vp, vp, vp, vp, i64, vp, vp, vp]),
    "drgb_fuzzy_weights_static": (C.c_int, [vp, vp, i64, i32, i32, vp, vp, vp, vp, i64, vp, vp, vp]),
    "drgb_find_ab": (C.c_int, [f32, f32, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "drgb_init_embedding": (C.c_int, [vp, i64, f32, u64, vp, vp]),
    "drgb_embed_epoch": (C.c_int, [vp, vp, vp, vp, vp, vp, i64, f32, f32, f32, i32, i32, u64, vp]),
    "drgb_embed_epochs": (C.c_int, [vp, vp, vp, vp, vp, vp, i64, f32, f32, f32, i32, i32, i32, i32,
                                    u64, vp]),
    "drgb_fit_transform": (C.c_int, [vp, vp, i64, i32, C.POINTER(Params), vp, EPOCH_CB, vp, vp]),
    "drgb_default_params": (C.c_int, [C.POINTER(Params)]),
    "drgb_mlp_param_count": (C.c_int64, []),
    "drgb_mlp_init": (C.c_int, [vp, vp, i32, u64, vp]),
    "drgb_mlp_sample": (C.c_int, [vp, vp, vp, vp, i64, i64, i32, i32, C.c_uint32, u64, vp, vp]),
    "drgb_mlp_grad": (C.c_int, [vp, vp, vp, i64, i32, vp, i32, i32, f32, f32, vp, vp, vp]),
    "drgb_mlp_train": (C.c_int, [vp, vp, i64, i32, vp, vp, vp, i64, f32, f32, C.POINTER(MlpParams), vp, vp, vp,
                                 vp, vp]),
    "drgb_mlp_embed": (C.c_int, [vp, vp, vp, i64, i32, vp, vp]),
    "drgb_transform": (C.c_int, [vp, vp, vp, i64, vp, i64, i32, C.POINTER(Params), vp, vp]),
    "drgb_fit_transform_batched": (C.c_int, [vp, vp, C.POINTER(C.c_int64), i32, i32, C.POINTER(Params),
                                             C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), vp, vp]),
    "drgb_autotune_epoch": (C.c_int, [vp, vp, vp, vp, vp, i64, f32, f32, i32, i32, u64, i32,
                                      C.POINTER(C.c_int32), C.POINTER(C.c_float), vp]),
    "drgb_eval_recall": (C.c_int, [vp, vp, vp, i64, i32, i32, i64, C.POINTER(C.c_double), vp]),
    "drgb_eval_trust": (C.c_int, [vp, vp, vp, i64, i32, i32, i64, C.POINTER(C.c_double), vp]),
    "drgb_render": (C.c_int, [vp, vp, vp, i64, i32, i32, f32, f32, C.POINTER(C.c_float), C.POINTER(C.c_float),
                              C.POINTER(C.c_float), vp, vp]),
    "drgb_wait_selftest": (C.c_int, [vp, i64, i32, vp]),
    "drgb_spectral_init": (C.c_int, [vp, vp, vp, vp, i64, f32, u64, vp, C.POINTER(C.c_double), vp]),
    "drgb_pca": (C.c_int, [vp, vp, i64, i32, i32, vp, vp, vp, C.POINTER(C.c_double), vp]),
    "drgb_eval_recall_heldout": (C.c_int, [vp, vp, vp, i64, vp, vp, i64, i32, i32, i64, C.POINTER(C.c_double),
                                           vp]),
}

_lib = None


def load() -> C.CDLL:
    """Load libdrgb.so and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is not built; run `python -m paper_2603_04035_gb300.build` "
                "(or __graft_entry__.build()) first")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
