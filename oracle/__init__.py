"""FP64 CPU oracle for the CPWL approximation method (test infrastructure).

This package is the plain, slow, obviously correct reference that the CUDA
library is checked against.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py`` may import it.  It shares
no code with the CUDA library: the arithmetic lives in ``pwl_oracle.c`` (plain
C, compiled here with gcc, IEEE semantics, no FMA contraction), and this module
only marshals numpy arrays to it.

Function descriptors are plain dicts ``{"kind": str, "a": float, "b": float,
"p": [...]}`` with the kinds and parameter meanings of ``pwl_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pwl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

KINDS = {"gaussian": 0, "lorentzian": 1, "bessel_j0": 2, "poly": 3, "exp": 4, "sampled": 5}


class _Func(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad", ctypes.c_int32), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("p", ctypes.c_double * 8)]


def build(force: bool = False) -> str:
    """Compile ``pwl_oracle.c`` into ``_build/liboracle.so`` (gcc, -O2, no FMA
    contraction so x86 and Arm give the same bits)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        F = ctypes.POINTER(_Func)
        i64 = ctypes.c_int64
        sig = {
            "orc_f": (ctypes.c_double, [F, ctypes.c_double]),
            "orc_f2": (ctypes.c_double, [F, ctypes.c_double]),
            "orc_f_many": (None, [F, D, i64, D]),
            "orc_j0_one_term": (None, [F, D, i64, D]),
            "orc_density": (None, [F, i64, D]),
            "orc_cumulative": (None, [D, i64, ctypes.c_double, D]),
            "orc_invert": (ctypes.c_int, [D, D, i64, ctypes.c_double, ctypes.c_double, i64, D]),
            "orc_design": (ctypes.c_int, [F, i64, i64, D, D, D]),
            "orc_interp_values": (None, [F, D, i64, D]),
            "orc_gauss_legendre": (None, [ctypes.c_int, D, D]),
            "orc_load_vector": (None, [F, D, i64, ctypes.c_int, D]),
            "orc_gram": (None, [D, i64, D, D, D]),
            "orc_thomas": (None, [i64, D, D, D, D]),
            "orc_project_values": (None, [F, D, i64, ctypes.c_int, D]),
            "orc_eval": (None, [D, D, i64, D, D, i64]),
            "orc_eval_grad": (None, [D, D, i64, D, D, i64, D, D, D, D, D]),
            "orc_l2_error": (ctypes.c_double, [F, D, D, i64, ctypes.c_int, ctypes.c_int, D]),
            "orc_integral_abs_f2_pow": (ctypes.c_double, [F, ctypes.c_double, i64, ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _func(desc) -> _Func:
    f = _Func()
    f.kind = KINDS[desc["kind"]]
    f.a = float(desc["a"])
    f.b = float(desc["b"])
    if desc["kind"] == "sampled":
        # host samples (numpy, FP64); the struct keeps them alive
        s = np.ascontiguousarray(desc["samples"], dtype=np.float64)
        f._samples = s
        f.p[0] = float(s.size)
        f.p[1] = np.frombuffer(np.uint64(s.ctypes.data).tobytes(), dtype=np.float64)[0]
        return f
    p = list(desc.get("p", [])) + [0.0] * (8 - len(desc.get("p", [])))
    for i in range(8):
        f.p[i] = float(p[i])
    return f


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------------------
# f, f''
# ----------------------------------------------------------------------------
def f(desc, x):
    lib, F = _load(), _func(desc)
    xs = np.atleast_1d(_f64(x))
    return np.array([lib.orc_f(ctypes.byref(F), float(v)) for v in xs])


def f_many(desc, x) -> np.ndarray:
    """f at every point of x (one C call; same values as f())."""
    lib, F = _load(), _func(desc)
    xs = _f64(np.atleast_1d(x)).ravel()
    out = np.empty_like(xs)
    lib.orc_f_many(ctypes.byref(F), _dp(xs), xs.size, _dp(out))
    return out


def j0_one_term(desc, x) -> np.ndarray:
    """A sqrt(2/(pi z)) cos(z - pi/4), z = alpha x: the one-term asymptotic
    form of A J0(alpha x) that the paper times (Section V-C); desc is a
    bessel_j0 descriptor."""
    lib, F = _load(), _func(desc)
    xs = _f64(np.atleast_1d(x)).ravel()
    out = np.empty_like(xs)
    lib.orc_j0_one_term(ctypes.byref(F), _dp(xs), xs.size, _dp(out))
    return out


def f2(desc, x):
    lib, F = _load(), _func(desc)
    xs = np.atleast_1d(_f64(x))
    return np.array([lib.orc_f2(ctypes.byref(F), float(v)) for v in xs])


# ----------------------------------------------------------------------------
# design (Section III-B)
# ----------------------------------------------------------------------------
def density(desc, M: int) -> np.ndarray:
    lib, F = _load(), _func(desc)
    d = np.empty(M, np.float64)
    lib.orc_density(ctypes.byref(F), M, _dp(d))
    return d


def cumulative(d, delta: float) -> np.ndarray:
    lib = _load()
    d = _f64(d)
    G = np.empty(d.size + 1, np.float64)
    lib.orc_cumulative(_dp(d), d.size, float(delta), _dp(G))
    return G


def invert(d, G, a: float, b: float, N: int):
    lib = _load()
    d, G = _f64(d), _f64(G)
    knots = np.empty(N + 1, np.float64)
    rc = lib.orc_invert(_dp(d), _dp(G), d.size, float(a), float(b), N, _dp(knots))
    return knots, rc


def design(desc, N: int, M: int | None = None, return_aux: bool = False):
    """Knots of the nearly optimal partition T* with N intervals, density
    sampled on M cells (default 64 N)."""
    lib, F = _load(), _func(desc)
    M = 64 * N if M is None else M
    knots = np.empty(N + 1, np.float64)
    d = np.empty(M, np.float64)
    G = np.empty(M + 1, np.float64)
    rc = lib.orc_design(ctypes.byref(F), N, M, _dp(knots), _dp(d), _dp(G))
    if return_aux:
        return knots, {"rc": rc, "d": d, "G": G}
    return knots


# ----------------------------------------------------------------------------
# vertex values (Section II-B)
# ----------------------------------------------------------------------------
def interp_values(desc, knots) -> np.ndarray:
    lib, F = _load(), _func(desc)
    knots = _f64(knots)
    v = np.empty(knots.size, np.float64)
    lib.orc_interp_values(ctypes.byref(F), _dp(knots), knots.size - 1, _dp(v))
    return v


def gauss_legendre(Q: int):
    lib = _load()
    x = np.empty(Q, np.float64)
    w = np.empty(Q, np.float64)
    lib.orc_gauss_legendre(Q, _dp(x), _dp(w))
    return x, w


def load_vector(desc, knots, Q: int = 8) -> np.ndarray:
    lib, F = _load(), _func(desc)
    knots = _f64(knots)
    b = np.empty(knots.size, np.float64)
    lib.orc_load_vector(ctypes.byref(F), _dp(knots), knots.size - 1, Q, _dp(b))
    return b


def gram(knots):
    lib = _load()
    knots = _f64(knots)
    n = knots.size
    lo, di, up = (np.empty(n, np.float64) for _ in range(3))
    lib.orc_gram(_dp(knots), n - 1, _dp(lo), _dp(di), _dp(up))
    return lo, di, up


def thomas(lower, diag, upper, rhs) -> np.ndarray:
    lib = _load()
    lower, diag, upper = _f64(lower), _f64(diag), _f64(upper)
    x = np.array(rhs, dtype=np.float64, copy=True)
    lib.orc_thomas(x.size, _dp(lower), _dp(diag), _dp(upper), _dp(x))
    return x


def project_values(desc, knots, Q: int = 8) -> np.ndarray:
    lib, F = _load(), _func(desc)
    knots = _f64(knots)
    c = np.empty(knots.size, np.float64)
    lib.orc_project_values(ctypes.byref(F), _dp(knots), knots.size - 1, Q, _dp(c))
    return c


def values(desc, knots, form: str, Q: int = 8) -> np.ndarray:
    if form == "interp":
        return interp_values(desc, knots)
    if form == "project":
        return project_values(desc, knots, Q)
    raise ValueError(form)


# ----------------------------------------------------------------------------
# evaluation (Algorithm 1) and gradients
# ----------------------------------------------------------------------------
def evaluate(knots, vals, x) -> np.ndarray:
    lib = _load()
    knots, vals = _f64(knots), _f64(vals)
    x = _f64(x).reshape(-1)
    y = np.empty_like(x)
    lib.orc_eval(_dp(knots), _dp(vals), knots.size - 1, _dp(x), _dp(y), x.size)
    return y


def evaluate_grad(knots, vals, x, gy):
    """Returns gx, gv, gxk, gv_abs, gxk_abs (the *_abs arrays hold sums of the
    absolute values of the accumulated terms, for error bounds)."""
    lib = _load()
    knots, vals = _f64(knots), _f64(vals)
    x = _f64(x).reshape(-1)
    gy = _f64(gy).reshape(-1)
    n = knots.size
    gx = np.empty_like(x)
    gv, gxk, gva, gxa = (np.zeros(n, np.float64) for _ in range(4))
    lib.orc_eval_grad(_dp(knots), _dp(vals), n - 1, _dp(x), _dp(gy), x.size, _dp(gx), _dp(gv),
                      _dp(gxk), _dp(gva), _dp(gxa))
    return gx, gv, gxk, gva, gxa


# ----------------------------------------------------------------------------
# error measures
# ----------------------------------------------------------------------------
def l2_error(desc, knots, vals, Q: int = 16, sub: int = 1, per_interval: bool = False):
    lib, F = _load(), _func(desc)
    knots, vals = _f64(knots), _f64(vals)
    n = knots.size
    per = np.empty(n, np.float64) if per_interval else None
    e = lib.orc_l2_error(ctypes.byref(F), _dp(knots), _dp(vals), n - 1, Q, sub,
                         _dp(per) if per is not None else None)
    return (e, per) if per_interval else e


def integral_abs_f2_pow(desc, p: float, n: int = 20000, Q: int = 16) -> float:
    lib, F = _load(), _func(desc)
    return lib.orc_integral_abs_f2_pow(ctypes.byref(F), float(p), n, Q)
