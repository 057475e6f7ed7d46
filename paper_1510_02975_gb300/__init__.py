"""GB300-native evaluation of nearly optimal continuous piecewise-linear
(CPWL) approximations (Berjon et al., "Optimal Piecewise Linear Function
Approximation for GPU-based Applications").

Thin binding over the C ABI of libpwl.so (include/pwl.h).  The functions
named like the C entry points take torch CUDA tensors, pass their pointers
and the current stream, and raise PwlError on a non-zero status.  PyTorch is
used only for device memory and streams; every step runs in the library's
CUDA kernels.  There is no CPU fallback: without a built library or a GPU
these functions raise.
"""
from __future__ import annotations

import ctypes

from ._capi import (DTYPES, FORMS, KINDS, PRECISIONS, PwlBatchInfo, PwlError, PwlFunc, PwlTableInfo, check, load,
                    make_func)

__all__ = [
    "PwlError", "pwl_design", "pwl_project", "pwl_table_build", "pwl_table_update", "pwl_table_check", "pwl_table_destroy", "pwl_table_get_info",
    "pwl_eval", "pwl_eval_variant", "pwl_eval_synthetic", "pwl_eval_synthetic_variant", "pwl_direct_eval",
    "pwl_direct_synthetic", "pwl_eval_backward", "pwl_eval_backward_noalloc",
    "pwl_error_constants", "pwl_predicted_error", "pwl_n_for_error",
    "pwl_batch_create", "pwl_batch_destroy", "pwl_batch_design", "pwl_batch_project", "pwl_batch_build",
    "pwl_batch_check", "pwl_batch_plan", "pwl_batch_eval", "pwl_batch_autotune", "pwl_batch_get_info", "Batch",
    "pwl_channels_forward", "pwl_channels_backward", "ChannelPWL", "pwl_test_fail_allocations",
    "pwl_batch_inject_wait_timeout", "Table", "design", "project", "PWLFunction",
    "KINDS", "FORMS", "DTYPES", "PRECISIONS",
]


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _require(t, dtype, name, numel=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype} (got {t.dtype})")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements (got {t.numel()})")


def _workspace(nbytes: int, device):
    torch = _torch()
    # 256-byte aligned: the caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


# ----------------------------------------------------------------------------
# C entry points, same names
# ----------------------------------------------------------------------------
def pwl_design(f, n_intervals: int, m_cells: int = 0, precision: str = "fp64", knots=None,
               workspace=None, stream=None):
    """Knots of the nearly optimal partition (Section III-B) -> float64 (N+1,)."""
    torch = _torch()
    lib = load()
    if knots is None:
        knots = torch.empty(n_intervals + 1, dtype=torch.float64, device="cuda")
    _require(knots, torch.float64, "knots", n_intervals + 1)
    ws_n = lib.pwl_design_workspace_size(n_intervals, m_cells)
    ws = workspace if workspace is not None and workspace.numel() >= ws_n else _workspace(ws_n, knots.device)
    F = make_func(f)
    check(lib.pwl_design(ctypes.byref(F), n_intervals, m_cells, PRECISIONS[precision], _ptr(knots),
                         _ptr(ws), ws.numel(), _stream(stream)), "pwl_design")
    return knots


def pwl_project(f, knots, form: str = "project", quad_points: int = 8, precision: str = "fp64",
                values=None, workspace=None, stream=None):
    """Vertex values of pi_T f ("interp") or P_T f ("project") -> float64 (N+1,)."""
    torch = _torch()
    lib = load()
    _require(knots, torch.float64, "knots")
    n = knots.numel() - 1
    if values is None:
        values = torch.empty_like(knots)
    _require(values, torch.float64, "values", n + 1)
    ws_n = lib.pwl_project_workspace_size(n)
    ws = workspace if workspace is not None and workspace.numel() >= ws_n else _workspace(ws_n, knots.device)
    F = make_func(f)
    check(lib.pwl_project(ctypes.byref(F), _ptr(knots), n, FORMS[form], quad_points, PRECISIONS[precision],
                          _ptr(values), _ptr(ws), ws.numel(), _stream(stream)), "pwl_project")
    return values


def pwl_table_build(knots, values, value_dtype: str = "fp32", k_cells: int = 0, stream=None):
    """Opaque table handle (int) for FP64 knots and values (synchronizes)."""
    torch = _torch()
    lib = load()
    _require(knots, torch.float64, "knots")
    _require(values, torch.float64, "values", knots.numel())
    out = ctypes.c_void_p()
    check(lib.pwl_table_build(_ptr(knots), _ptr(values), knots.numel() - 1, DTYPES[value_dtype], k_cells,
                              ctypes.byref(out), _stream(stream)), "pwl_table_build")
    return out.value


def pwl_table_update(handle, knots, values, stream=None) -> None:
    """Asynchronous in-place rebuild from new FP64 knots / values (same N)."""
    torch = _torch()
    _require(knots, torch.float64, "knots")
    _require(values, torch.float64, "values", knots.numel())
    check(load().pwl_table_update(ctypes.c_void_p(handle), _ptr(knots), _ptr(values), _stream(stream)),
          "pwl_table_update")


def pwl_table_check(handle, stream=None) -> None:
    check(load().pwl_table_check(ctypes.c_void_p(handle), _stream(stream)), "pwl_table_check")


def pwl_table_destroy(handle) -> None:
    if handle:
        check(load().pwl_table_destroy(ctypes.c_void_p(handle)), "pwl_table_destroy")


def pwl_table_get_info(handle) -> dict:
    info = PwlTableInfo()
    check(load().pwl_table_get_info(ctypes.c_void_p(handle), ctypes.byref(info)), "pwl_table_get_info")
    return {k: getattr(info, k) for k, _ in PwlTableInfo._fields_}


def _io_dtype(t):
    torch = _torch()
    return {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}[t.dtype]


def pwl_eval(handle, x, y=None, stream=None):
    """y = v(x) (Algorithm 1); x, y float32 / bfloat16 / float16 CUDA tensors."""
    torch = _torch()
    if y is None:
        y = torch.empty_like(x)
    if x.dtype != y.dtype or x.numel() != y.numel():
        raise ValueError("x and y must have the same dtype and size")
    if not (x.is_cuda and y.is_cuda and x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y must be contiguous CUDA tensors")
    check(load().pwl_eval(ctypes.c_void_p(handle), _ptr(x), _ptr(y), x.numel(), _io_dtype(x), _stream(stream)),
          "pwl_eval")
    return y


def pwl_eval_variant(handle, mode: int, x, y=None, stream=None):
    """Comparison paths: mode 0 binary search (Algorithm 1), mode 1 texture filter."""
    torch = _torch()
    _require(x, torch.float32, "x")
    if y is None:
        y = torch.empty_like(x)
    _require(y, torch.float32, "y", x.numel())
    check(load().pwl_eval_variant(ctypes.c_void_p(handle), mode, _ptr(x), _ptr(y), x.numel(), _stream(stream)),
          "pwl_eval_variant")
    return y


def pwl_eval_synthetic(handle, m: int, seed: int = 0, out=None, stream=None):
    """Compute-ceiling run: Algorithm 1 on m queries generated in registers;
    returns (or adds into `out`) the float64 checksum of the results."""
    torch = _torch()
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
    _require(out, torch.float64, "out", 1)
    check(load().pwl_eval_synthetic(ctypes.c_void_p(handle), int(seed) & 0xFFFFFFFF, int(m), _ptr(out),
                                    _stream(stream)), "pwl_eval_synthetic")
    return out


def pwl_eval_synthetic_variant(handle, mode: int, m: int, seed: int = 0, out=None, stream=None):
    """pwl_eval_synthetic for the comparison paths of pwl_eval_variant (modes 0..5)."""
    torch = _torch()
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
    _require(out, torch.float64, "out", 1)
    check(load().pwl_eval_synthetic_variant(ctypes.c_void_p(handle), int(mode), int(seed) & 0xFFFFFFFF, int(m),
                                            _ptr(out), _stream(stream)), "pwl_eval_synthetic_variant")
    return out


DIRECT_METHODS = {"library": 0, "fast": 1}


def pwl_direct_eval(f, method: str, x, y=None, stream=None):
    """y = f(x) evaluated directly in FP32 (the paper's comparison systems):
    method "library" (expf, IEEE division, j0f) or "fast" (__expf,
    __fdividef, the one-term asymptotic J0 with __cosf and rsqrtf)."""
    torch = _torch()
    _require(x, torch.float32, "x")
    if y is None:
        y = torch.empty_like(x)
    _require(y, torch.float32, "y", x.numel())
    F = make_func(f)
    check(load().pwl_direct_eval(ctypes.byref(F), DIRECT_METHODS[method], _ptr(x), _ptr(y), x.numel(),
                                 _stream(stream)), "pwl_direct_eval")
    return y


def pwl_direct_synthetic(f, method: str, m: int, seed: int = 0, out=None, stream=None):
    """Compute ceiling of pwl_direct_eval: f at m register-generated queries;
    returns (or adds into `out`) the float64 checksum."""
    torch = _torch()
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
    _require(out, torch.float64, "out", 1)
    F = make_func(f)
    check(load().pwl_direct_synthetic(ctypes.byref(F), DIRECT_METHODS[method], int(seed) & 0xFFFFFFFF, int(m),
                                      _ptr(out), _stream(stream)), "pwl_direct_synthetic")
    return out


def pwl_error_constants(f, m_cells: int = 0, out=None, stream=None):
    """The integrals of |f''|^{2/5} and f''^2 over [a, b] (Results 4-6),
    midpoint rule on m_cells cells -> float64 (2,) on the GPU."""
    torch = _torch()
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device="cuda")
    _require(out, torch.float64, "out", 2)
    F = make_func(f)
    check(load().pwl_error_constants(ctypes.byref(F), int(m_cells), _ptr(out), _stream(stream)),
          "pwl_error_constants")
    return out


def pwl_predicted_error(int_f2_25: float, int_f2_sq: float, a: float, b: float, n_intervals: int,
                        form: str = "interp", uniform: bool = False) -> float:
    """Predicted L2 error with N intervals (Results 4-6)."""
    r = ctypes.c_double()
    check(load().pwl_predicted_error(float(int_f2_25), float(int_f2_sq), float(a), float(b), int(n_intervals),
                                     FORMS[form], int(bool(uniform)), ctypes.byref(r)), "pwl_predicted_error")
    return r.value


def pwl_n_for_error(int_f2_25: float, int_f2_sq: float, a: float, b: float, target_l2: float,
                    form: str = "interp", uniform: bool = False) -> int:
    """Smallest N whose predicted L2 error is <= target_l2 (Results 4-6)."""
    r = ctypes.c_int64()
    check(load().pwl_n_for_error(float(int_f2_25), float(int_f2_sq), float(a), float(b), float(target_l2),
                                 FORMS[form], int(bool(uniform)), ctypes.byref(r)), "pwl_n_for_error")
    return r.value


def pwl_eval_backward(handle, x, gy, gx=None, g_values=None, g_knots=None, workspace=None, stream=None):
    """Backward of pwl_eval: returns gx; accumulates into g_values / g_knots."""
    torch = _torch()
    lib = load()
    _require(x, torch.float32, "x")
    _require(gy, torch.float32, "gy", x.numel())
    if gx is None:
        gx = torch.empty_like(x)
    _require(gx, torch.float32, "gx", x.numel())
    for name, t in (("g_values", g_values), ("g_knots", g_knots)):
        if t is not None:
            _require(t, torch.float32, name)
    need = lib.pwl_eval_backward_workspace_size(ctypes.c_void_p(handle))
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, x.device)
    check(lib.pwl_eval_backward(ctypes.c_void_p(handle), _ptr(x), _ptr(gy), _ptr(gx), _ptr(g_values),
                                _ptr(g_knots), x.numel(), _ptr(workspace), workspace.numel(), _stream(stream)),
          "pwl_eval_backward")
    return gx


def pwl_eval_backward_noalloc(handle, x, gy, gx=None, g_values=None, g_knots=None, stream=None):
    """pwl_eval_backward without a workspace: the partial sums go to the
    library's static device array (for callers that cannot allocate; calls
    that overlap on the GPU race)."""
    torch = _torch()
    _require(x, torch.float32, "x")
    _require(gy, torch.float32, "gy", x.numel())
    if gx is None:
        gx = torch.empty_like(x)
    _require(gx, torch.float32, "gx", x.numel())
    check(load().pwl_eval_backward_noalloc(ctypes.c_void_p(handle), _ptr(x), _ptr(gy), _ptr(gx), _ptr(g_values),
                                           _ptr(g_knots), x.numel(), _stream(stream)), "pwl_eval_backward_noalloc")
    return gx


def pwl_batch_create(funcs, n_intervals, m_per_interval: int = 0, cells_per_knot: int = 0):
    """Opaque batch handle (int) for F function descriptors and their N_f."""
    lib = load()
    F = len(funcs)
    if len(n_intervals) != F:
        raise ValueError("one n_intervals entry per function")
    arr = (PwlFunc * max(F, 1))()
    for i, f in enumerate(funcs):
        arr[i] = make_func(f)
    ns = (ctypes.c_int64 * max(F, 1))(*[int(n) for n in n_intervals])
    out = ctypes.c_void_p()
    check(lib.pwl_batch_create(arr, ns, F, m_per_interval, cells_per_knot, ctypes.byref(out)), "pwl_batch_create")
    return out.value


def pwl_batch_destroy(handle) -> None:
    if handle:
        check(load().pwl_batch_destroy(ctypes.c_void_p(handle)), "pwl_batch_destroy")


def pwl_batch_design(handle, precision: str = "fp64", stream=None) -> None:
    check(load().pwl_batch_design(ctypes.c_void_p(handle), PRECISIONS[precision], _stream(stream)),
          "pwl_batch_design")


def pwl_batch_project(handle, form: str = "project", quad_points: int = 8, precision: str = "fp64",
                      stream=None) -> None:
    check(load().pwl_batch_project(ctypes.c_void_p(handle), FORMS[form], quad_points, PRECISIONS[precision],
                                   _stream(stream)), "pwl_batch_project")


def pwl_batch_build(handle, stream=None) -> None:
    check(load().pwl_batch_build(ctypes.c_void_p(handle), _stream(stream)), "pwl_batch_build")


def pwl_batch_check(handle, stream=None) -> None:
    check(load().pwl_batch_check(ctypes.c_void_p(handle), _stream(stream)), "pwl_batch_check")


def pwl_batch_plan(handle, query_offsets, shape: int = -1, stage_min: int = -1) -> None:
    """query_offsets: F+1 non-decreasing ints (host sequence), first 0."""
    qo = (ctypes.c_int64 * len(query_offsets))(*[int(q) for q in query_offsets])
    check(load().pwl_batch_plan(ctypes.c_void_p(handle), qo, shape, stage_min), "pwl_batch_plan")


def pwl_batch_eval(handle, x, y=None, stream=None):
    torch = _torch()
    _require(x, torch.float32, "x")
    planned = pwl_batch_get_info(handle)["total_queries"]
    if x.numel() < planned:
        raise ValueError(f"x has {x.numel()} elements; the plan has {planned} queries")
    if y is None:
        y = torch.empty_like(x)
    _require(y, torch.float32, "y", x.numel())
    check(load().pwl_batch_eval(ctypes.c_void_p(handle), _ptr(x), _ptr(y), _stream(stream)), "pwl_batch_eval")
    return y


def pwl_batch_autotune(handle, x, y, reps: int = 3, stream=None) -> dict:
    """Times every (shape, stage_min) candidate, keeps the fastest plan and
    returns {(shape, stage_min): mean ms per launch}."""
    torch = _torch()
    _require(x, torch.float32, "x")
    planned = pwl_batch_get_info(handle)["total_queries"]
    if x.numel() < planned:
        raise ValueError(f"x has {x.numel()} elements; the plan has {planned} queries")
    _require(y, torch.float32, "y", x.numel())
    t = (ctypes.c_float * 20)()
    check(load().pwl_batch_autotune(ctypes.c_void_p(handle), _ptr(x), _ptr(y), reps, t, _stream(stream)),
          "pwl_batch_autotune")
    return {(shape, stage_min): float(t[4 * shape + j])
            for shape in range(5) for j, stage_min in enumerate((0, 4, 16, 64))}


def pwl_test_fail_allocations(succeed_first: int) -> None:
    """Failure injection: the next succeed_first device allocations of the
    library succeed and later ones fail with PWL_ENOMEM (< 0 resets)."""
    check(load().pwl_test_fail_allocations(int(succeed_first)), "pwl_test_fail_allocations")


def pwl_batch_inject_wait_timeout(handle, withhold: bool, wait_limit_ns: int = 0) -> None:
    """Failure injection: the asynchronous batch shape's staging waits run out
    after wait_limit_ns (withhold=True); withhold=False restores them."""
    check(load().pwl_batch_inject_wait_timeout(ctypes.c_void_p(handle), int(bool(withhold)), int(wait_limit_ns)),
          "pwl_batch_inject_wait_timeout")


def pwl_batch_get_info(handle) -> dict:
    info = PwlBatchInfo()
    check(load().pwl_batch_get_info(ctypes.c_void_p(handle), ctypes.byref(info)), "pwl_batch_get_info")
    return {k: getattr(info, k) for k, _ in PwlBatchInfo._fields_}


def pwl_channels_forward(knots, values, x, y=None, k_cells: int = 0, status=None, stream=None):
    """y[r, c] = v_c(x[r, c]); knots, values float32 [C, N+1]; x [R, C] float32 or bfloat16."""
    torch = _torch()
    _require(knots, torch.float32, "knots")
    _require(values, torch.float32, "values", knots.numel())
    C, n1 = knots.shape
    if x.dim() != 2 or x.shape[1] != C or not x.is_contiguous() or not x.is_cuda:
        raise ValueError("x must be a contiguous CUDA tensor [rows, C]")
    if y is None:
        y = torch.empty_like(x)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=x.device)
    io = {torch.float32: 0, torch.bfloat16: 1}[x.dtype]
    check(load().pwl_channels_forward(_ptr(knots), _ptr(values), C, n1 - 1, k_cells, _ptr(x), _ptr(y), x.shape[0],
                                      io, _ptr(status), _stream(stream)), "pwl_channels_forward")
    return y


def pwl_channels_backward(knots, values, x, gy, gx=None, g_values=None, g_knots=None, k_cells: int = 0,
                          status=None, stream=None):
    """Backward of pwl_channels_forward (FP32): returns gx; accumulates g_values, g_knots [C, N+1]."""
    torch = _torch()
    _require(knots, torch.float32, "knots")
    _require(values, torch.float32, "values", knots.numel())
    C, n1 = knots.shape
    _require(x, torch.float32, "x")
    _require(gy, torch.float32, "gy", x.numel())
    if gx is None:
        gx = torch.empty_like(x)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=x.device)
    check(load().pwl_channels_backward(_ptr(knots), _ptr(values), C, n1 - 1, k_cells, _ptr(x), _ptr(gy), _ptr(gx),
                                       _ptr(g_values), _ptr(g_knots), x.shape[0], _ptr(status), _stream(stream)),
          "pwl_channels_backward")
    return gx


# ----------------------------------------------------------------------------
# convenience layer
# ----------------------------------------------------------------------------
def design(f, n_intervals: int, m_cells: int = 0, precision: str = "fp64"):
    return pwl_design(f, n_intervals, m_cells, precision)


def project(f, knots, form: str = "project", quad_points: int = 8, precision: str = "fp64"):
    return pwl_project(f, knots, form, quad_points, precision)


class Table:
    """A CPWL function on the GPU (owns a pwl_table)."""

    def __init__(self, knots, values, value_dtype: str = "fp32", k_cells: int = 0):
        self.handle = pwl_table_build(knots, values, value_dtype, k_cells)
        self.info = pwl_table_get_info(self.handle)
        self.n_intervals = int(self.info["n_intervals"])

    def __call__(self, x, out=None):
        return pwl_eval(self.handle, x, out)

    def eval(self, x, out=None):
        return pwl_eval(self.handle, x, out)

    def variant(self, mode: int, x, out=None):
        return pwl_eval_variant(self.handle, mode, x, out)

    def update(self, knots, values):
        pwl_table_update(self.handle, knots, values)

    def backward(self, x, gy, gx=None, g_values=None, g_knots=None):
        return pwl_eval_backward(self.handle, x, gy, gx, g_values, g_knots)

    def close(self):
        if getattr(self, "handle", None):
            pwl_table_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent CPWL functions on the GPU (owns a pwl_batch)."""

    def __init__(self, funcs, n_intervals, m_per_interval: int = 0, cells_per_knot: int = 0):
        self.handle = pwl_batch_create(funcs, n_intervals, m_per_interval, cells_per_knot)
        self.n_funcs = len(funcs)
        self.n_intervals = [int(n) for n in n_intervals]

    def design(self, precision: str = "fp64", stream=None):
        pwl_batch_design(self.handle, precision, stream)

    def project(self, form: str = "project", quad_points: int = 8, precision: str = "fp64", stream=None):
        pwl_batch_project(self.handle, form, quad_points, precision, stream)

    def build(self, stream=None):
        pwl_batch_build(self.handle, stream)

    def check(self, stream=None):
        pwl_batch_check(self.handle, stream)

    def plan(self, query_offsets, shape: int = -1, stage_min: int = -1):
        pwl_batch_plan(self.handle, query_offsets, shape, stage_min)

    def eval(self, x, out=None, stream=None):
        return pwl_batch_eval(self.handle, x, out, stream)

    def autotune(self, x, y, reps: int = 3):
        return pwl_batch_autotune(self.handle, x, y, reps)

    def info(self) -> dict:
        return pwl_batch_get_info(self.handle)

    def _device_array(self, key, typestr, copy):
        """The batch's concatenated device array `key` as a torch tensor:
        a copy, or (copy=False) a view that the next design / projection /
        build overwrites and that pwl_batch_destroy frees."""
        torch = _torch()
        info = self.info()

        class _Cai:
            __cuda_array_interface__ = {"shape": (int(info["total_knots"]),), "typestr": typestr,
                                        "data": (int(info[key]), False), "version": 3}

        t = torch.as_tensor(_Cai(), device="cuda")
        return t.clone() if copy else t

    def knots(self, copy: bool = True):
        """float64 knots of all functions; function f's at offsets()[f]."""
        return self._device_array("d_knots", "<f8", copy)

    def values(self, copy: bool = True):
        return self._device_array("d_values", "<f8", copy)

    def knots_fp32(self, copy: bool = True):
        return self._device_array("d_knots_fp32", "<f4", copy)

    def values_fp32(self, copy: bool = True):
        return self._device_array("d_values_fp32", "<f4", copy)

    def offsets(self):
        out = [0]
        for n in self.n_intervals:
            out.append(out[-1] + n + 1)
        return out

    def close(self):
        if getattr(self, "handle", None):
            pwl_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_FUNCS = {}


def _autograd_classes():
    """torch.autograd.Function subclasses, defined on first use."""
    if _FUNCS:
        return _FUNCS
    torch = _torch()

    class _TableFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, handle, g_values, g_knots):
            ctx.save_for_backward(x)
            ctx.handle, ctx.gv, ctx.gk = handle, g_values, g_knots
            return pwl_eval(handle, x.contiguous())

        @staticmethod
        def backward(ctx, gy):
            (x,) = ctx.saved_tensors
            gx = pwl_eval_backward(ctx.handle, x.contiguous(), gy.contiguous(), None, ctx.gv, ctx.gk)
            return gx, None, None, None

    class _ChannelFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, knots, values, k_cells, k_cells_bwd, status):
            ctx.save_for_backward(x, knots, values)
            ctx.k_cells_bwd, ctx.status = k_cells_bwd, status
            return pwl_channels_forward(knots, values, x.contiguous(), k_cells=k_cells, status=status)

        @staticmethod
        def backward(ctx, gy):
            x, knots, values = ctx.saved_tensors
            gv = torch.zeros_like(values) if ctx.needs_input_grad[2] else None
            gk = torch.zeros_like(knots) if ctx.needs_input_grad[1] else None
            # the backward kernel takes FP32 streams: a BF16 map's x and gy
            # are widened (exactly) and gx is returned in x's dtype
            gx = pwl_channels_backward(knots, values, x.contiguous().float(), gy.contiguous().float(), None, gv, gk,
                                       k_cells=ctx.k_cells_bwd, status=ctx.status)
            return gx.to(x.dtype), gk, gv, None, None, None

    _FUNCS["table"] = _TableFn
    _FUNCS["channels"] = _ChannelFn
    return _FUNCS


class PWLFunction:
    """y = v(x) through a Table with autograd: gradients flow to x; if
    table_grads = (g_values, g_knots) FP32 tensors of N+1 are given, the
    backward accumulates the table gradients into them."""

    @staticmethod
    def apply(table: Table, x, table_grads=None):
        gv, gk = table_grads if table_grads is not None else (None, None)
        return _autograd_classes()["table"].apply(x, table.handle, gv, gk)


class ChannelPWL:
    """Channel-wise learnable CPWL map with autograd: y[r, c] = v_c(x[r, c])
    for x [R, C] (float32 or bfloat16), knots and values [C, N+1] (float32
    leaf tensors).  The backward gives gradients w.r.t. x (in x's dtype), the
    values and the knots.

    status: an int32 CUDA tensor of one element that the forward and backward
    kernels OR their status bits into (bit 0: a channel's knots are not
    strictly increasing, e.g. after a training step crossed two knots; the
    results of that step are then unspecified).  The caller zeroes it and
    reads it with ChannelPWL.check(status) between steps, where a host
    synchronisation costs nothing; None gives each call a status word that
    nothing reads."""

    @staticmethod
    def apply(x, knots, values, k_cells: int = 0, k_cells_backward: int = 0, status=None):
        return _autograd_classes()["channels"].apply(x, knots, values, k_cells, k_cells_backward, status)

    @staticmethod
    def new_status(device="cuda"):
        return _torch().zeros(1, dtype=_torch().int32, device=device)

    @staticmethod
    def check(status) -> None:
        """Raises PwlError (PWL_EINVAL) if a kernel set a status bit since the
        word was zeroed (synchronizes with the device)."""
        bits = int(status.item())
        if bits & 1:
            raise PwlError(1, "ChannelPWL", "a channel's knots are not strictly increasing")
        if bits:
            raise PwlError(1, "ChannelPWL", f"status bits {bits:#x}")
