"""ctypes binding of libspsvm.so: the C ABI of include/spsvm.h, name for
name, with argument marshalling only (torch tensors -> raw device
pointers, Python numbers -> C scalars).  Every computation runs in the
library's CUDA kernels; there is no Python or CPU fallback, and loading
fails loudly if the library is missing or cannot be built."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))

SPSVM_OK = 0
SPSVM_ERR_ARG = -1
SPSVM_ERR_OOM = -2
SPSVM_ERR_NOT_PD = -3
SPSVM_ERR_NO_CONVERGE = -4
SPSVM_ERR_CUDA = -5
SPSVM_ERR_TIMEOUT = -6
SPSVM_ERR_BUSY = -7

SPSVM_FP32 = 0
SPSVM_BF16SPLIT = 1
SPSVM_SOLVE_MIXED = 0
SPSVM_SOLVE_FP64 = 1
SPSVM_GROWTH_EPS_PAPER = 5e-6
SPSVM_SCORE_HEURISTIC = 0
SPSVM_SCORE_EXACT = 1

PRECISIONS = {"fp32": SPSVM_FP32, "bf16split": SPSVM_BF16SPLIT}


class spsvm_kmat(C.Structure):
    _fields_ = [("data", C.c_void_p), ("format", C.c_int32), ("pad_", C.c_int32),
                ("n", C.c_int64), ("rows", C.c_int64), ("ld", C.c_int64),
                ("plane", C.c_int64)]


class spsvm_points(C.Structure):
    _fields_ = [("X", C.c_void_p), ("n", C.c_int64), ("d", C.c_int64), ("ldx", C.c_int64),
                ("norms", C.c_void_p), ("hi", C.c_void_p), ("lo", C.c_void_p),
                ("ldh", C.c_int64), ("mid", C.c_void_p)]


class spsvm_options(C.Structure):
    _fields_ = [("candidates", C.c_int32), ("add_per_round", C.c_int32),
                ("max_newton", C.c_int32), ("precision", C.c_int32),
                ("growth_tol", C.c_double), ("rel_tol", C.c_double),
                ("seed", C.c_uint64), ("initial_basis", C.POINTER(C.c_int64)),
                ("n_initial", C.c_int32), ("fixed_basis", C.c_int32),
                ("refine", C.c_int32), ("record", C.c_int32), ("stream", C.c_void_p),
                ("newton_solver", C.c_int32), ("score", C.c_int32), ("bias", C.c_int32),
                ("lowrank", C.c_int32)]


class spsvm_problem(C.Structure):
    _fields_ = [("rows", C.c_void_p), ("n_rows", C.c_int64), ("y", C.c_void_p),
                ("gamma", C.c_float), ("pad_", C.c_float), ("lambda_", C.c_double),
                ("basis_budget", C.c_int32), ("pad2_", C.c_int32), ("tol", C.c_double),
                ("seed", C.c_uint64)]


class spsvm_step(C.Structure):
    _fields_ = [("basis", C.c_int32), ("active", C.c_int32), ("gnorm", C.c_double),
                ("t", C.c_double), ("loss", C.c_double), ("errors", C.c_int32),
                ("jitter", C.c_int32), ("changed", C.c_int32), ("solve", C.c_int32)]


SPSVM_NEWTON_NONE = 0
SPSVM_NEWTON_FACTOR = 1
SPSVM_NEWTON_REUSE = 2
SPSVM_NEWTON_LOWRANK = 3
SPSVM_LOWRANK_KMAX = 128


_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_F = C.c_float
_D = C.c_double
_SZ = C.c_size_t

# name -> (restype, argtypes); the full list of exported entry points.
SIGNATURES = {
    "spsvm_prepare_points": (_I32, [C.POINTER(spsvm_points), _I32, _P]),
    "spsvm_kernel_block_scratch_bytes": (_SZ, [_I64, _I64, _I32]),
    "spsvm_kernel_block": (_I32, [C.POINTER(spsvm_points), _P, _I32, _F, _I32,
                                  C.POINTER(spsvm_kmat), _I64, _P, _SZ, _P]),
    "spsvm_score_scratch_bytes": (_SZ, [_I64, _I64, _I32]),
    "spsvm_score_candidates": (_I32, [C.POINTER(spsvm_points), _P, _P, _P, _I32, _F, _D, _I32,
                                      _P, _P, _P, _P, _SZ, _P]),
    "spsvm_score_candidates_noalloc": (_I32, [C.POINTER(spsvm_points), _P, _P, _P, _I32, _F, _D,
                                              _I32, _P, _P, _P, _P]),
    "spsvm_reduce_scratch_bytes": (_SZ, [_I64]),
    "spsvm_outputs": (_I32, [C.POINTER(spsvm_kmat), _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "spsvm_gemv": (_I32, [C.POINTER(spsvm_kmat), _P, _P, _I32, _P]),
    "spsvm_compact_scratch_bytes": (_SZ, [_I64, _I64]),
    "spsvm_compact_active": (_I32, [C.POINTER(spsvm_kmat), _P, _P, _P, _P, _P,
                                    C.POINTER(spsvm_kmat), _P, _P, _P, _SZ, _P]),
    "spsvm_gram_scratch_bytes": (_SZ, [_I64, _I64]),
    "spsvm_gram": (_I32, [C.POINTER(spsvm_kmat), _P, _I64, C.POINTER(spsvm_kmat), _P, _D, _I32,
                          _P, _I64, _P, _SZ, _P]),
    "spsvm_cholesky_work_bytes": (_SZ, [_I64]),
    "spsvm_cholesky": (_I32, [_P, _I64, _I64, _P, _P, _SZ, _P]),
    "spsvm_cholesky_solve_work_bytes": (_SZ, [_I64]),
    "spsvm_mixed_work_bytes": (_SZ, [_I64]),
    "spsvm_cholesky_mixed": (_I32, [_P, _I64, _I64, C.c_double, _P, _P, _SZ, _P]),
    "spsvm_solve_mixed": (_I32, [_P, _I64, _I64, C.c_double, _P, _P, _I32, C.c_double,
                                 C.POINTER(_I32), C.POINTER(C.c_double), _P, _SZ, _P]),
    "spsvm_cholesky_solve": (_I32, [_P, _I64, _I64, _P, _P, _SZ, _P]),
    "spsvm_active_diff": (_I32, [C.POINTER(spsvm_kmat), _P, _P, _I32, _P, _I64, _P, _P, _P, _SZ,
                                 _P]),
    "spsvm_lowrank_work_bytes": (_SZ, [_I64, _I32]),
    "spsvm_lowrank_factor": (_I32, [_P, _SZ, _I64, _P, _I64, _P, _I32, _P, _SZ, _P, _P]),
    "spsvm_solve_lowrank": (_I32, [_P, _I64, _I64, _P, _P, _I32, C.c_double, C.POINTER(_I32),
                                   C.POINTER(C.c_double), _P, _SZ, _P, _SZ, _I32, _P]),
    "spsvm_line_scratch_bytes": (_SZ, [_I64]),
    "spsvm_line_search": (_I32, [_P, _P, _P, _I64, _P, _P, _I32, _D, C.POINTER(_D), _P, _P, _SZ,
                                 _P]),
    "spsvm_decision_scratch_bytes": (_SZ, [_I64, _I64, _I64, _I32]),
    "spsvm_decision": (_I32, [_P, _I64, _I64, _P, _P, _I64, _I64, _I64, _F, _I32, _P, _P, _SZ,
                              _P]),
    "spsvm_fit_workspace_bytes": (_SZ, [_I64, _I64, _I32, C.POINTER(spsvm_options)]),
    "spsvm_fit": (_I32, [_P, _I64, _I64, _I64, _P, _F, _D, _I32, _D, C.POINTER(spsvm_options),
                         _P, _SZ, C.POINTER(_P)]),
    "spsvm_predict": (_I32, [_P, _P, _I64, _I64, _P, _P]),
    "spsvm_predict_work_bytes": (_SZ, [_P, _I64]),
    "spsvm_predict_ws": (_I32, [_P, _P, _I64, _I64, _P, _P, _SZ, _P]),
    "spsvm_model_info": (_I32, [_P, C.POINTER(_I32), C.POINTER(_I64), C.POINTER(_F),
                                C.POINTER(_D), C.POINTER(_D), C.POINTER(_I32), C.POINTER(_I32),
                                C.POINTER(_I32)]),
    "spsvm_model_get": (_I32, [_P, _P, _P]),
    "spsvm_model_history": (_I32, [_P, _P, _I32, C.POINTER(_I32)]),
    "spsvm_model_round": (_I32, [_P, _I32, _P, C.POINTER(_I32), _P, C.POINTER(_I32)]),
    "spsvm_model_outputs": (_I32, [_P, _P, _I64]),
    "spsvm_free": (None, [_P]),
    "spsvm_draw_candidates": (_I32, [_I64, _P, _I32, _I32, C.c_uint64, C.c_uint32, _P]),
    "spsvm_fit_batched": (_I32, [_P, _I64, _I64, _I64, C.POINTER(spsvm_problem), _I32,
                                 C.POINTER(spsvm_options), _I32, _P, _P]),
    "spsvm_score_exact_scratch_bytes": (_SZ, [_I64, _I64, _I32, _I32]),
    "spsvm_score_candidates_exact": (_I32, [C.POINTER(spsvm_points), _P, _P, _P, _I32, _F,
                                            C.c_double, _I32, _P, _P, _P, _P, _SZ, _P]),
    "spsvm_model_bias": (_I32, [_P, C.POINTER(C.c_double)]),
    "spsvm_fit_ovo": (_I32, [_P, _I64, _I64, _I64, _P, _I32, _F, C.c_double, _I32, C.c_double,
                             C.POINTER(spsvm_options), _I32, _P, _P]),
    "spsvm_predict_ovo_work_bytes": (_SZ, [_I32, _I64]),
    "spsvm_predict_ovo": (_I32, [_P, _I32, _P, _I64, _I64, _P, _P, _P, _SZ, _P]),
    "spsvm_server_create": (_I32, [_SZ, _I32, C.POINTER(_P)]),
    "spsvm_server_submit_fit": (_I32, [_P, _P, _I64, _I64, _P, _F, _D, _I32, _D,
                                       C.POINTER(spsvm_options), C.POINTER(_I64)]),
    "spsvm_server_submit_predict": (_I32, [_P, _I64, _P, _I64, C.POINTER(_I64)]),
    "spsvm_server_wait": (_I32, [_P, _I64, _D, C.POINTER(_I32), C.POINTER(_D)]),
    "spsvm_server_result": (_I32, [_P, _I64, _P, _I64, C.POINTER(_P)]),
    "spsvm_server_stats": (_I32, [_P, C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_SZ),
                                  C.POINTER(_SZ)]),
    "spsvm_server_destroy": (None, [_P]),
    "spsvm_server_release": (_I32, [_P, _I64]),
    "spsvm_model_device_bytes": (_SZ, [_P]),
    "spsvm_launch_count": (C.c_uint64, []),
    "spsvm_profile_enable": (_I32, [_I32]),
    "spsvm_profile_read": (_I32, [_I32, C.POINTER(C.c_char_p), C.POINTER(_I64), C.POINTER(_D),
                                  C.POINTER(_D)]),
    "spsvm_device_status": (_I32, [C.POINTER(_I32)]),
    "spsvm_stream_status": (_I32, [_P, C.POINTER(_I32)]),
    "spsvm_set_wait_limit": (None, [C.c_uint32]),
    "spsvm_set_factor_ctas": (None, [C.c_uint32]),
    "spsvm_strerror": (C.c_char_p, [_I32]),
    "spsvm_last_error": (C.c_char_p, []),
    "spsvm_version": (C.c_char_p, []),
}

_lib = None


def lib_path():
    return os.path.join(_HERE, "_build", "libspsvm.so")


def load(build_if_missing: bool = True):
    """Loads libspsvm.so (building it with nvcc first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if build_if_missing:
        from . import build as _b
        path = _b.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libspsvm.so not found at {path}; run paper_1404_1066_gb300.build")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SpsvmError(RuntimeError):
    def __init__(self, code, where):
        lib = load(False)
        msg = lib.spsvm_last_error().decode(errors="replace")
        super().__init__(f"{where}: {lib.spsvm_strerror(code).decode()} ({code}): {msg}")
        self.code = code


def check(code, where):
    if code != SPSVM_OK:
        raise SpsvmError(code, where)
    return code


def ptr(t):
    """Raw pointer of a torch tensor (device or host), or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream
