"""ctypes declarations of libcoot.so (include/coot.h).  Argument
marshalling only: every step of the computation runs inside the library."""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_uint, c_uint64, c_void_p

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libcoot.so")

COOT_F32, COOT_BF16, COOT_F16, COOT_F64, COOT_I32, COOT_U32 = 0, 1, 2, 3, 4, 5
COOT_NORM_INF, COOT_NORM_NEG_INF, COOT_NORM_FRO = -1, -2, -3
HEAD_SUM, HEAD_SUMSQ, HEAD_NORM2, HEAD_SUMABS = 1, 2, 4, 8
HEAD_MIN, HEAD_MAX, HEAD_MINABS, HEAD_MAXABS = 16, 32, 64, 128
HEAD_ALL, HEAD_ANY = 256, 512
HEAD_COLSUM, HEAD_ROWSUM = 1024, 2048
STAT_SUM, STAT_MEAN, STAT_VAR, STAT_STDDEV, STAT_MIN, STAT_MAX = 1, 2, 4, 8, 16, 32
KIND_MAP, KIND_REDUCE, KIND_COLSUM, KIND_ROWSUM, KIND_BATCHED = 0, 1, 2, 3, 4
KIND_COLSTATS, KIND_ROWSTATS, KIND_MULTI, KIND_DIMS = 5, 6, 7, 8

STATUS = ["COOT_OK", "COOT_ERR_INVALID_ARG", "COOT_ERR_BAD_TREE", "COOT_ERR_SHAPE", "COOT_ERR_DTYPE",
          "COOT_ERR_ALIAS", "COOT_ERR_EMPTY", "COOT_ERR_UNSUPPORTED", "COOT_ERR_COMPILE", "COOT_ERR_CUDA",
          "COOT_ERR_TIMEOUT", "COOT_ERR_NOT_INIT", "COOT_ERR_WORKSPACE"]


class coot_mat(ctypes.Structure):
    _fields_ = [("ptr", c_void_p), ("dtype", c_int32), ("reserved", c_int32),
                ("n_rows", c_int64), ("n_cols", c_int64), ("ld", c_int64)]


_u8p = c_char_p      # tree bytes
_matp = POINTER(coot_mat)
_dp = c_void_p       # device double*

# name -> (restype, argtypes); every function in include/coot.h
SIGNATURES = {
    "coot_init": (c_int, [c_int, c_uint]),
    "coot_finalize": (c_int, []),
    "coot_last_error": (c_char_p, []),
    "coot_status_string": (c_char_p, [c_int]),
    "coot_version": (c_int, []),
    "coot_workspace_size": (c_int, [c_int64, POINTER(c_size_t)]),
    "coot_tree_check": (c_int, [_u8p, c_size_t, POINTER(c_int), POINTER(c_int), POINTER(c_uint64)]),
    "coot_tree_compile": (c_int, [_u8p, c_size_t, c_int, c_int, c_int, c_uint, c_char_p, POINTER(c_size_t)]),
    "coot_tree_source": (c_int, [_u8p, c_size_t, c_int, c_char_p, c_size_t, POINTER(c_size_t)]),
    "coot_expr_eval": (c_int, [_u8p, c_size_t, _matp, c_int, _matp, c_void_p, c_size_t, c_void_p]),
    "coot_accu": (c_int, [_u8p, c_size_t, _matp, c_int, _dp, c_void_p, c_size_t, c_void_p]),
    "coot_sum_dim": (c_int, [_u8p, c_size_t, _matp, c_int, c_int, _matp, c_void_p, c_size_t, c_void_p]),
    "coot_dot": (c_int, [_matp, _matp, _dp, c_void_p, c_size_t, c_void_p]),
    "coot_norm": (c_int, [_u8p, c_size_t, _matp, c_int, c_int, _dp, c_void_p, c_size_t, c_void_p]),
    "coot_minmax": (c_int, [_u8p, c_size_t, _matp, c_int, _dp, c_void_p, c_size_t, c_void_p]),
    "coot_all_any": (c_int, [_u8p, c_size_t, _matp, c_int, _dp, c_void_p, c_size_t, c_void_p]),
    "coot_set_canonical": (c_int, [c_int]),
    "coot_device_status": (c_int, [POINTER(c_int)]),
    "coot_host_device_pointer": (c_int, [c_void_p, POINTER(c_void_p)]),
    "coot_submat": (c_int, [_matp, c_int64, c_int64, c_int64, c_int64, _matp]),
    "coot_diag": (c_int, [_matp, c_int64, _matp]),
    "coot_tree_canonical": (c_int, [_u8p, c_size_t, c_void_p, c_size_t, POINTER(c_size_t)]),
    "coot_stats_dim": (c_int, [_u8p, c_size_t, _matp, c_int, c_int, c_uint, c_int, _matp, c_void_p, c_size_t,
                               c_void_p]),
    "coot_expr_reduce": (c_int, [_u8p, c_size_t, _matp, c_int, c_uint, _matp, _dp, c_void_p, c_size_t, c_void_p]),
    "coot_expr_multi": (c_int, [POINTER(c_void_p), POINTER(c_size_t), c_int, _matp, c_int, _matp, POINTER(c_uint),
                                _dp, c_void_p, c_size_t, c_void_p]),
    "coot_expr_multi_dims": (c_int, [POINTER(c_void_p), POINTER(c_size_t), c_int, _matp, c_int, _matp,
                                     POINTER(c_uint), _dp, _matp, _matp, c_void_p, c_size_t, c_void_p]),
    "coot_unfused_tmp_count": (c_int, [_u8p, c_size_t, POINTER(c_int)]),
    "coot_unfused_eval": (c_int, [_u8p, c_size_t, _matp, c_int, _matp, c_void_p, c_size_t, c_void_p]),
}


class CootError(RuntimeError):
    def __init__(self, func: str, status: int, message: str):
        self.func = func
        self.status = status
        self.status_name = STATUS[status] if 0 <= status < len(STATUS) else f"status {status}"
        super().__init__(f"{func}: {self.status_name}: {message}")


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded library.  Raises ImportError if it has not been built:
    there is no other implementation to fall back to."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with `python -m paper_2308_03120_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def call(name: str, *args) -> None:
    """Call an ABI function and raise CootError on a non-OK status."""
    L = lib()
    status = getattr(L, name)(*args)
    if status != 0:
        raise CootError(name, status, (L.coot_last_error() or b"").decode(errors="replace"))


class coot_batch_item(ctypes.Structure):
    _fields_ = [("in_", c_void_p * 4), ("ld_in", c_int64 * 4), ("out", c_void_p), ("ld_out", c_int64),
                ("colsum", c_void_p), ("ld_colsum", c_int64), ("n_rows", c_int64), ("n_cols", c_int64)]


_itemp = POINTER(coot_batch_item)
SIGNATURES.update({
    "coot_batch_plan_size": (c_int, [_itemp, c_int, POINTER(c_size_t), POINTER(c_int64)]),
    "coot_batch_plan_build": (c_int, [_itemp, c_int, c_int, c_void_p, c_size_t]),
    "coot_expr_eval_batched": (c_int, [_u8p, c_size_t, POINTER(c_int32), c_int32, c_int32, c_void_p, c_int,
                                       c_int64, c_void_p]),
})

SIGNATURES["coot_sum_rows_f32_static"] = (c_int, [_matp, _matp, c_void_p])

SIGNATURES["coot_set_launch_config"] = (c_int, [c_int, c_int, c_int, c_int, c_int, c_int64])
SIGNATURES["coot_last_launch"] = (c_int, [POINTER(c_int), POINTER(c_int), POINTER(c_int), POINTER(c_int64),
                                          POINTER(c_int64)])

# learned launch shapes
MODEL_FEATURES, MODEL_HIDDEN = 21, 64
POLICY_BUILTIN, POLICY_LEARNED = 0, 1
_fp = c_void_p  # float* (device or host buffer address)
SIGNATURES.update({
    "coot_mlp_forward": (c_int, [_fp, c_int, c_int, _fp, c_int, _fp, _fp, c_void_p]),
    "coot_mlp_loss_grad": (c_int, [_fp, c_int, c_int, _fp, _fp, c_int, _fp, _fp, _fp, _fp, _fp, c_void_p]),
    "coot_mlp_adam": (c_int, [_fp, _fp, _fp, _fp, c_int, c_int, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, c_void_p]),
    "coot_call_features": (c_int, [_u8p, c_size_t, c_int, POINTER(c_int32), c_int, c_uint, c_int64, c_int64, c_int,
                                   c_int, c_int, c_int, c_int64, POINTER(ctypes.c_float)]),
    "coot_model_load": (c_int, [POINTER(ctypes.c_float), c_size_t]),
    "coot_model_predict": (c_int, [POINTER(ctypes.c_float), c_int, POINTER(ctypes.c_float)]),
    "coot_set_policy": (c_int, [c_int]),
    "coot_launch_candidates": (c_int, [c_int, POINTER(c_int32), c_int, POINTER(c_int)]),
    "coot_prepare": (c_int, [_u8p, c_size_t, c_int, POINTER(c_int32), c_int, c_uint, c_int, c_int, c_int]),
})
