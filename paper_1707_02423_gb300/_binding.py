"""ctypes binding of libcfsim.so (include/cfsim.h): argument marshalling only.

Every computation happens in the library's kernels.  Loading fails loudly
when the library has not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

# The library this process loads: libcfsim.so beside this file, or another
# build of it named by CFSIM_LIBRARY (e.g. the debug-bounds build,
# libcfsim_debug.so, from build.build(variant="debug_bounds")).
LIB_PATH = os.environ.get("CFSIM_LIBRARY") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcfsim.so")

CF_OK = 0
CF_NORM_FROB = 0
CF_NORM_NONE = 1
CF_MATCH_GREEDY = 0
CF_MATCH_OPTIMAL = 1
CF_FLAG_PER_PAIR_LAUNCH = 1
CF_FLAG_PLAN_ONLY = 2
CF_FLAG_REUSE_PLAN = 4
CF_FLAG_OPT_UNSTAGED = 8
CF_FLAG_PER_PAIR_STREAMS = 16
CF_PROBE_SMEM, CF_PROBE_L2, CF_PROBE_DSMEM, CF_PROBE_FP32 = 0, 1, 2, 3
CF_DIST_SCALE01 = 1
DIST_NAMES = ("euclidean", "manhattan", "minkowski", "jaccard", "cosine")


class cf_cfg_view(C.Structure):
    _fields_ = [("n_blocks", C.c_int32), ("n_edges", C.c_int32), ("src", C.c_void_p), ("dst", C.c_void_p),
                ("w", C.c_void_p), ("attr", C.c_void_p)]


class cf_params(C.Structure):
    _fields_ = [("alpha", C.c_float), ("K", C.c_int32), ("norm_mode", C.c_int32), ("match_mode", C.c_int32),
                ("flags", C.c_uint32), ("tune", C.c_int32)]


class cf_probe_result(C.Structure):
    _fields_ = [("work", C.c_double), ("best_ms", C.c_double), ("rate", C.c_double), ("sm_mhz", C.c_double),
                ("per_clk_sm", C.c_double), ("n_sm", C.c_int32)]


class cf_tune_info(C.Structure):
    _fields_ = [("tune", C.c_int32), ("threads_per_cta", C.c_int32), ("smallest_group", C.c_int32),
                ("matching", C.c_int32), ("cluster", C.c_int32)]


class cf_pack_info(C.Structure):
    _fields_ = [("n_cfgs", C.c_int32), ("F", C.c_int32), ("F_pad", C.c_int32), ("max_blocks", C.c_int32),
                ("n_blocks", C.c_int64), ("n_edges", C.c_int64), ("n_user_edges", C.c_int64), ("bytes", C.c_int64)]


_p = C.c_void_p
_i32 = C.c_int32
_i64p = C.POINTER(C.c_int64)
_szp = C.POINTER(C.c_size_t)

# name -> (restype, argtypes); the exported surface of include/cfsim.h
SIGNATURES = {
    "cf_status_string": (C.c_char_p, [_i32]),
    "cf_last_error_detail": (C.c_char_p, []),
    "cf_abi_version": (_i32, []),
    "cf_pack_size": (_i32, [_p, _i32, _i32, _szp]),
    "cf_pack_host": (_i32, [_p, _i32, _i32, _p, C.c_size_t]),
    "cf_pack_info_get": (_i32, [_p, C.POINTER(cf_pack_info)]),
    "cf_pack_cfgs": (_i32, [_p, _i32, _i32, _p, C.c_size_t, _p]),
    "cf_pack_set_weights": (_i32, [_p, _p, _p, _p]),
    "cf_out_sizes": (_i32, [_p, _p, _p, _i32, _i64p, _i64p]),
    "cf_similarity_ws_size": (_i32, [_p, _p, _p, _i32, C.POINTER(cf_params), _szp]),
    "cf_similarity": (_i32, [_p, _p, _p, _i32, C.POINTER(cf_params), _p, _p, _p, _p, _p, C.c_size_t, _p]),
    "cf_match": (_i32, [_p, _p, _p, _i32, C.POINTER(cf_params), _p, _p, _p, _p, _p, C.c_size_t, _p]),
    "cf_similarity_backward_ws_size": (_i32, [_p, _p, _p, _i32, C.POINTER(cf_params), _szp]),
    "cf_similarity_backward": (_i32, [_p, _p, _p, _i32, C.POINTER(cf_params), _p, _p, _p, _p, _p, _p, _p,
                                      C.c_size_t, _p]),
    "cf_topk": (_i32, [_p, _i32, _i32, _i32, _p, _p, _p]),
    "cf_topk_pairs": (_i32, [_p, _i32, _i32, _p, _p, _p]),
    "cf_similarity_ws_size_any": (_i32, [_p, _p, _i32, C.POINTER(cf_params), _szp]),
    "cf_similarity_noalloc": (_i32, [_p, _p, _p, _i32, C.POINTER(cf_params), _p, _p, _p, _p, _p, _p]),
    "cf_status_check": (_i32, [_p, _p]),
    "cf_distances_ws_size": (_i32, [_i32, _szp]),
    "cf_distances": (_i32, [_p, _p, _p, _i32, C.c_float, C.c_uint32, _p, _p, C.c_size_t, _p]),
    "cf_score_matrix": (_i32, [_p, _p, _i32, _i32, _i32, _i32, _p, _p, _p]),
    "cf_ward_ws_size": (_i32, [_i32, _szp]),
    "cf_ward": (_i32, [_p, _i32, _i32, _p, _p, _p, _p, C.c_size_t, _p]),
    "cf_num_tunes": (_i32, []),
    "cf_tune_describe": (_i32, [_i32, C.POINTER(cf_tune_info)]),
    "cf_autotune_ws_size": (_i32, [_p, _p, _p, _i32, C.POINTER(cf_params), _szp]),
    "cf_autotune": (_i32, [_p, _p, _p, _p, _p, _i32, C.POINTER(cf_params), _p, _p, C.c_size_t, C.c_char_p, _p,
                           C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
    "cf_graph_begin": (_i32, [_p]),
    "cf_graph_end": (_i32, [_p, C.POINTER(C.c_void_p)]),
    "cf_graph_launch": (_i32, [_p, _p]),
    "cf_graph_nodes": (_i32, [_p]),
    "cf_graph_destroy": (_i32, [_p]),
    "cf_probe_ws_size": (_i32, [_i32, _szp]),
    "cf_probe": (_i32, [_i32, _p, C.c_size_t, _i32, _p, C.POINTER(cf_probe_result)]),
}


class CfsimError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"cfsim status {status}: {message}")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """Load libcfsim.so once (after torch, so that its CUDA runtime is the one
    the library binds to) and declare every exported signature."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise CfsimError(-1, f"{LIB_PATH} is not built; call paper_1707_02423_gb300.build.build() first")
        import torch  # noqa: F401  (loads the CUDA runtime the library links against)

        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int) -> None:
    if status != CF_OK:
        L = lib()
        msg = L.cf_status_string(status).decode()
        detail = L.cf_last_error_detail().decode()
        raise CfsimError(status, f"{msg}: {detail}" if detail else msg)


def params(alpha: float = 0.8, K: int = 40, norm_mode: int = CF_NORM_FROB, flags: int = 0, tune: int = 0,
           match_mode: int = CF_MATCH_GREEDY) -> cf_params:
    return cf_params(float(alpha), int(K), int(norm_mode), int(match_mode), int(flags), int(tune))
