"""ctypes view of the C ABI declared in include/pwl.h (libpwl.so).

Only argument marshalling lives here.  Loading fails loudly when the shared
library has not been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

PWL_OK, PWL_EINVAL, PWL_ENOMEM, PWL_ECUDA, PWL_ENOTSUP, PWL_ETIMEOUT = range(6)
KINDS = {"gaussian": 0, "lorentzian": 1, "bessel_j0": 2, "poly": 3, "exp": 4, "sampled": 5}
FORMS = {"interp": 0, "project": 1}
DTYPES = {"fp32": 0, "bf16": 1, "fp16": 2}
PRECISIONS = {"fp64": 0, "fp32": 1}
STATUS_NAMES = {0: "PWL_OK", 1: "PWL_EINVAL", 2: "PWL_ENOMEM", 3: "PWL_ECUDA", 4: "PWL_ENOTSUP",
                5: "PWL_ETIMEOUT"}


class PwlError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class PwlFunc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("p", ctypes.c_double * 8)]


class PwlTableInfo(ctypes.Structure):
    _fields_ = [("n_intervals", ctypes.c_int64), ("k_cells", ctypes.c_int64), ("n_chain", ctypes.c_int64),
                ("value_dtype", ctypes.c_int32), ("reserved", ctypes.c_int32), ("a", ctypes.c_float),
                ("b", ctypes.c_float), ("d_knots", ctypes.c_void_p), ("d_values", ctypes.c_void_p),
                ("eval_smem_bytes", ctypes.c_size_t), ("backward_smem_bytes", ctypes.c_size_t),
                ("layout", ctypes.c_int32), ("reserved2", ctypes.c_int32)]


class PwlBatchInfo(ctypes.Structure):
    _fields_ = [("n_funcs", ctypes.c_int64), ("total_knots", ctypes.c_int64), ("total_cells", ctypes.c_int64),
                ("index_bytes", ctypes.c_int64), ("total_queries", ctypes.c_int64), ("eval_grid", ctypes.c_int32),
                ("eval_threads", ctypes.c_int32), ("eval_shape", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("n_items", ctypes.c_int64), ("n_staged", ctypes.c_int64), ("stage_min", ctypes.c_int64),
                ("smem_bytes", ctypes.c_int64), ("d_knot_offsets", ctypes.c_void_p), ("d_knots", ctypes.c_void_p),
                ("d_values", ctypes.c_void_p), ("d_knots_fp32", ctypes.c_void_p),
                ("d_values_fp32", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_SZ = ctypes.c_size_t
_ST = ctypes.c_int

# name -> (restype, argtypes); every symbol include/pwl.h declares
SIGNATURES = {
    "pwl_last_error": (ctypes.c_char_p, []),
    "pwl_version": (_I32, []),
    "pwl_func_sampled": (_ST, [ctypes.c_double, ctypes.c_double, _P, _I64, ctypes.POINTER(PwlFunc)]),
    "pwl_design_workspace_size": (_SZ, [_I64, _I64]),
    "pwl_design": (_ST, [ctypes.POINTER(PwlFunc), _I64, _I64, _I32, _P, _P, _SZ, _P]),
    "pwl_project_workspace_size": (_SZ, [_I64]),
    "pwl_project": (_ST, [ctypes.POINTER(PwlFunc), _P, _I64, _I32, _I32, _I32, _P, _P, _SZ, _P]),
    "pwl_table_build": (_ST, [_P, _P, _I64, _I32, _I64, ctypes.POINTER(_P), _P]),
    "pwl_table_update": (_ST, [_P, _P, _P, _P]),
    "pwl_table_check": (_ST, [_P, _P]),
    "pwl_table_destroy": (_ST, [_P]),
    "pwl_table_get_info": (_ST, [_P, ctypes.POINTER(PwlTableInfo)]),
    "pwl_eval": (_ST, [_P, _P, _P, _I64, _I32, _P]),
    "pwl_eval_variant": (_ST, [_P, _I32, _P, _P, _I64, _P]),
    "pwl_eval_synthetic": (_ST, [_P, ctypes.c_uint32, _I64, _P, _P]),
    "pwl_eval_synthetic_variant": (_ST, [_P, _I32, ctypes.c_uint32, _I64, _P, _P]),
    "pwl_direct_eval": (_ST, [ctypes.POINTER(PwlFunc), _I32, _P, _P, _I64, _P]),
    "pwl_direct_synthetic": (_ST, [ctypes.POINTER(PwlFunc), _I32, ctypes.c_uint32, _I64, _P, _P]),
    "pwl_error_constants": (_ST, [ctypes.POINTER(PwlFunc), _I64, _P, _P]),
    "pwl_predicted_error": (_ST, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _I64, _I32, _I32, ctypes.POINTER(ctypes.c_double)]),
    "pwl_n_for_error": (_ST, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _I32, _I32, ctypes.POINTER(_I64)]),
    "pwl_eval_backward_workspace_size": (_SZ, [_P]),
    "pwl_eval_backward": (_ST, [_P, _P, _P, _P, _P, _P, _I64, _P, _SZ, _P]),
    "pwl_eval_backward_noalloc": (_ST, [_P, _P, _P, _P, _P, _P, _I64, _P]),
    "pwl_batch_create": (_ST, [ctypes.POINTER(PwlFunc), ctypes.POINTER(_I64), _I64, _I64, _I64,
                               ctypes.POINTER(_P)]),
    "pwl_batch_destroy": (_ST, [_P]),
    "pwl_batch_design": (_ST, [_P, _I32, _P]),
    "pwl_batch_project": (_ST, [_P, _I32, _I32, _I32, _P]),
    "pwl_batch_build": (_ST, [_P, _P]),
    "pwl_batch_check": (_ST, [_P, _P]),
    "pwl_batch_plan": (_ST, [_P, ctypes.POINTER(_I64), _I32, _I64]),
    "pwl_batch_eval": (_ST, [_P, _P, _P, _P]),
    "pwl_batch_autotune": (_ST, [_P, _P, _P, _I32, ctypes.POINTER(ctypes.c_float), _P]),
    "pwl_batch_get_info": (_ST, [_P, ctypes.POINTER(PwlBatchInfo)]),
    "pwl_channels_forward": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _I64, _I32, _P, _P]),
    "pwl_channels_backward": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _P, _P, _P, _I64, _P, _P]),
    "pwl_test_fail_allocations": (_ST, [_I64]),
    "pwl_batch_inject_wait_timeout": (_ST, [_P, _I32, ctypes.c_uint64]),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load():
    """Load libpwl.so and declare its signatures.  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"libpwl.so not built ({path}); run __graft_entry__.build() or "
                              f"python -m paper_1510_02975_gb300._build")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int, where: str) -> None:
    if status != PWL_OK:
        msg = load().pwl_last_error()
        raise PwlError(status, where, msg.decode() if msg else "")


def make_func(desc) -> PwlFunc:
    if desc["kind"] == "sampled":
        # samples: a contiguous CUDA float64 tensor that the caller keeps alive
        smp = desc["samples"]
        if not (getattr(smp, "is_cuda", False) and str(smp.dtype) == "torch.float64" and smp.is_contiguous()):
            raise TypeError("samples must be a contiguous CUDA float64 tensor")
        f = PwlFunc()
        check(load().pwl_func_sampled(float(desc["a"]), float(desc["b"]), ctypes.c_void_p(smp.data_ptr()),
                                      smp.numel(), ctypes.byref(f)), "pwl_func_sampled")
        return f
    f = PwlFunc()
    f.kind = KINDS[desc["kind"]]
    f.reserved = 0
    f.a = float(desc["a"])
    f.b = float(desc["b"])
    p = list(desc.get("p", []))
    p += [0.0] * (8 - len(p))
    for i in range(8):
        f.p[i] = float(p[i])
    return f
