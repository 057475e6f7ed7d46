"""Helpers shared by the GPU parity tests: rounding of tables to the storage
types the library uses, and tolerances.

Tolerances (from the arithmetic):
  FP32 evaluation of the same CPWL table: |y - y_ref| <= 5e-7 max|y_ref|
    (the FP32 slope has relative error 2^-24, the FMA one more rounding:
     both <= 2^-24 |v_i - v_{i-1}| + 2^-24 |y|, well inside 5e-7 max|y|).
  FP64 design and projection: knots within 1e-12 (b - a); values within
    1e-12 max|v| (different summation orders and cyclic reduction vs Thomas).
  Table gradients (FP32 accumulation): within 1e-5 of the sum of the
    absolute values of the accumulated terms (FP64 reference).
  FP32 design mode (FP32 densities, compensated sums, FP64 scan and
    inversion): a relative density error eps moves knot i by about
    eps N (G(x_i) / G_M) h_i, so each knot is held within
    max(1e-3, 1e-6 N) of the shorter of its two intervals (eps up to ~1e-6:
    the FP32 f'' of J0 near its zeros).
  FP32 integrand mode of the vertex values: f is evaluated in FP32 at
    FP32-rounded points, so each f(t) carries |t f'(t)| 2^-24 from the
    argument plus the FP32 function's own error (below 2^-18 max|f| for the
    library J0); v_i = f(x_i) takes that once, and P_T's hat sums average it
    and the Gram solve (its diagonal scaling has off-diagonal row sums 1/2)
    at most doubles it: |v - v_ref| <= 2.5 env (fp32_integrand_envelope).
"""
import numpy as np

EVAL_REL = 5e-7
DESIGN_REL = 1e-12
VALUES_REL = 1e-12
GRAD_REL = 1e-5


def fp32_integrand_envelope(desc, samples: int = 20001) -> float:
    """max|f| 2^-18 + max|t f'(t)| 2^-24 over [a, b] (f from the oracle,
    f' by central differences on `samples` points)."""
    import oracle
    t = np.linspace(desc["a"], desc["b"], samples)
    ft = oracle.f_many(desc, t)
    return float(np.abs(ft).max() * 2.0 ** -18 + np.abs(t * np.gradient(ft, t)).max() * 2.0 ** -24)


def fp32_design_bound(ref_knots) -> np.ndarray:
    """Per-knot bound of the FP32 design mode against the FP64 oracle."""
    h = np.diff(ref_knots)
    h_adj = np.minimum(np.r_[h[0], h], np.r_[h, h[-1]])
    return max(1e-3, 1e-6 * h.size) * h_adj


def round_values(v, dtype: str) -> np.ndarray:
    """FP64 values -> FP32 (round to nearest) -> 16-bit type, widened back."""
    import torch
    v32 = np.asarray(v, dtype=np.float64).astype(np.float32)
    if dtype == "fp32":
        return v32.astype(np.float64)
    if dtype == "fp16":
        return v32.astype(np.float16).astype(np.float64)
    if dtype == "bf16":
        return torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
    raise ValueError(dtype)


def round_knots(k) -> np.ndarray:
    return np.asarray(k, dtype=np.float64).astype(np.float32).astype(np.float64)
