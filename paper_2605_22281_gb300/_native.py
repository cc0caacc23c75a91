"""ctypes mirror of include/sfl.h (argument marshalling only).

Loading fails loudly: if libsfl.so cannot be built or loaded, or the process has
no CUDA device when a compute call is made, a RuntimeError is raised.  There is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import builder as _build

SFL_OK, SFL_EINVAL, SFL_ENOMEM, SFL_ECUDA, SFL_ENONFINITE, SFL_ETIMEOUT, SFL_EUNSUPPORTED = range(7)
SFL_F64, SFL_F32, SFL_BF16 = 0, 1, 2
STOP_RUNNING, STOP_DISCREPANCY, STOP_MAXIT, STOP_BREAKDOWN = 0, 1, 2, 3
PRECOND = {"identity": 0, "diag": 1, "reweight": 2, "lowrank": 3}
STOP_RULE = {"residual": 0, "normal": 1}
SKETCH_APPLY = {"auto": 0, "fused": 1, "kernel": 2}
SKETCH_KIND = {"sparse_sign": 0, "srht": 1, "gaussian": 2}
DTYPE = {"f64": SFL_F64, "f32": SFL_F32, "bf16": SFL_BF16}


class Csr(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("values", ctypes.c_void_p),
                ("dtype", ctypes.c_int)]


class PlanOpts(ctypes.Structure):
    _fields_ = [("value_dtype", ctypes.c_int), ("lanes_per_row", ctypes.c_int32), ("max_device_bytes", ctypes.c_uint64),
                ("image_rows", ctypes.c_int32), ("image_cols", ctypes.c_int32), ("slot_layout", ctypes.c_int32),
                ("index_bits", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32), ("zeta", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("window", ctypes.c_int32), ("maxit", ctypes.c_int32), ("noise_norm", ctypes.c_double),
                ("eta", ctypes.c_double), ("precond", ctypes.c_int32), ("stop_rule", ctypes.c_int32),
                ("diag_w", ctypes.c_void_p), ("irw_eps", ctypes.c_double), ("vec_dtype", ctypes.c_int32),
                ("spmm_tile", ctypes.c_int32), ("x_history", ctypes.c_void_p), ("relres_history", ctypes.c_void_p),
                ("orth_against_z", ctypes.c_int32), ("sketch_dense", ctypes.c_void_p),
                ("sketch_dense_stop", ctypes.c_void_p), ("lowrank_rank", ctypes.c_int32),
                ("lowrank_oversample", ctypes.c_int32), ("lowrank_power", ctypes.c_int32),
                ("lowrank_omega", ctypes.c_void_p), ("lowrank_fp64", ctypes.c_int32),
                ("sketch_apply", ctypes.c_int32), ("sketch_kind", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("relres", ctypes.c_double),
                ("tol", ctypes.c_double)]


class KernelTimes(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 12), ("launches", ctypes.c_int32 * 12)]


KERNEL_CLASSES = ["sketch_init", "init_b", "init_bwd", "orth_z", "spmv_fwd", "orth_w", "spmv_bwd", "small_ls",
                  "solution", "sketch", "orth_full", "lowrank"]


class PlanStats(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("nnz_A", ctypes.c_int64),
                ("nnz_At", ctypes.c_int64), ("padded_nnz_A", ctypes.c_int64), ("padded_nnz_At", ctypes.c_int64),
                ("lanes_A", ctypes.c_int32), ("lanes_At", ctypes.c_int32), ("value_dtype", ctypes.c_int32),
                ("unmatched", ctypes.c_int32), ("device_bytes", ctypes.c_uint64), ("tiled_At", ctypes.c_int32),
                ("matrix_free", ctypes.c_int32), ("index_bytes_A", ctypes.c_int32), ("index_bytes_At", ctypes.c_int32)]


class CtGeometry(ctypes.Structure):
    _fields_ = [("image_n", ctypes.c_int32), ("n_angles", ctypes.c_int32), ("n_bins", ctypes.c_int32),
                ("back", ctypes.c_int32), ("angles_cs", ctypes.c_void_p)]


_P = ctypes.c_void_p
_SIGNATURES = {
    "sfl_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(Csr), ctypes.POINTER(Csr),
                                        ctypes.POINTER(PlanOpts), _P]),
    "sfl_plan_destroy": (ctypes.c_int, [_P]),
    "sfl_plan_create_ct": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(CtGeometry), ctypes.POINTER(PlanOpts), _P]),
    "sfl_plan_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(PlanStats)]),
    "sfl_plan_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "sflsqr_solve": (ctypes.c_int, [_P, _P, ctypes.POINTER(Opts), _P, ctypes.POINTER(Info), _P]),
    "sflsmr_solve": (ctypes.c_int, [_P, _P, ctypes.POINTER(Opts), _P, ctypes.POINTER(Info), _P]),
    "sflsqr_solve_host": (ctypes.c_int, [_P, _P, ctypes.POINTER(Opts), _P, ctypes.POINTER(Info), _P]),
    "sflsmr_solve_host": (ctypes.c_int, [_P, _P, ctypes.POINTER(Opts), _P, ctypes.POINTER(Info), _P]),
    "flsqr_solve": (ctypes.c_int, [_P, _P, ctypes.POINTER(Opts), _P, ctypes.POINTER(Info), _P]),
    "flsqr_solve_host": (ctypes.c_int, [_P, _P, ctypes.POINTER(Opts), _P, ctypes.POINTER(Info), _P]),
    "sfl_solve_host_loop": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(Opts), _P, ctypes.POINTER(Info), _P]),
    "sfl_solve_profiled": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(Opts), _P, ctypes.POINTER(Info),
                                          ctypes.POINTER(KernelTimes), _P]),
    "sfl_sketch_export": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, _P, _P]),
    "sfl_sketch_apply": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int64, _P, _P]),
    "sfl_sketch_apply_noalloc": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int64,
                                                _P, _P]),
    "sflsqr_solve_batched": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.POINTER(Opts), _P, _P, _P]),
    "sfl_batched_tile": (ctypes.c_int, [_P, ctypes.c_int32]),
    "sflsqr_fixed_batched": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.POINTER(Opts), _P, _P, _P]),
    "sflsqr_adjoint_batched": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, _P, _P]),
    "sfl_fixed_calls": (ctypes.c_int64, [_P]),
    "sfl_error_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sfl_last_cuda_error": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsfl.so (building it first if needed) and declare the signatures."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libsfl.so not found at {path}; run paper_2605_22281_gb300.build.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class SflError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.sfl_error_string(status).decode()
        detail = lib.sfl_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} ({status})" + (f" [{detail}]" if detail else ""))
        self.status = status


def check(status: int, where: str) -> None:
    if status != SFL_OK:
        raise SflError(status, where)
