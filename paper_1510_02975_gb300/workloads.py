"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input recipes only (function descriptors, query streams,
parameter draws) and none of the method's arithmetic; the CUDA path, the
oracle-based tests and the benchmark all draw their inputs from here.

Function descriptors are dicts {"kind", "a", "b", "p"} with the meaning of
pwl_func in include/pwl.h:
  gaussian   p = (A, mu, s):  A exp(-(x-mu)^2 / (2 s^2))
  lorentzian p = (A, x0, g):  A / (1 + ((x-x0)/g)^2)
  bessel_j0  p = (A, alpha):  A J0(alpha x)
"""
from __future__ import annotations

import math

import numpy as np

# The three functions of the paper's experiments (Sections V-A, V-B, V-C) on
# the domains used here: the Gaussian exp(-x^2/2) on [-4, 4], the
# Lorentzian 1/(1+x^2) on [-10, 10] and J0 on [0, 50].
GAUSSIAN = {"kind": "gaussian", "a": -4.0, "b": 4.0, "p": [1.0, 0.0, 1.0]}
LORENTZIAN = {"kind": "lorentzian", "a": -10.0, "b": 10.0, "p": [1.0, 0.0, 1.0]}
BESSEL_J0 = {"kind": "bessel_j0", "a": 0.0, "b": 50.0, "p": [1.0, 1.0]}
PAPER_FUNCTIONS = {"gaussian": GAUSSIAN, "lorentzian": LORENTZIAN, "bessel_j0": BESSEL_J0}

# small case: the Gaussian with 64 knots (63 intervals), 10^6 uniform queries
SMALL = {"func": GAUSSIAN, "n_intervals": 63, "m": 10**6, "seed": 0}
# at scale: the three functions x N in {256, 1024, 4096} intervals, two query
# sets of 2^28 each: uniform on the domain (seed 1) and normal(0, 1.5)
# clipped to the domain (seed 2)
SCALE_N = (256, 1024, 4096)
SCALE_M = 1 << 28


def uniform_queries(desc, m: int, seed: int, device="cuda", dtype=None):
    """m float32 queries uniform on [a, b) (torch Philox stream of `seed`)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.rand(m, generator=g, device=device, dtype=torch.float32)
    x.mul_(float(desc["b"] - desc["a"])).add_(float(desc["a"]))
    return x if dtype is None else x.to(dtype)


def lowbias32(v):
    """The 32-bit integer hash "lowbias32" (hash-prospector project), on a
    numpy uint32 array: xor-shift 16, multiply 0x7feb352d, xor-shift 15,
    multiply 0x846ca68b, xor-shift 16 (all mod 2^32)."""
    v = np.asarray(v, dtype=np.uint32).copy()
    v ^= v >> np.uint32(16)
    v *= np.uint32(0x7FEB352D)
    v ^= v >> np.uint32(15)
    v *= np.uint32(0x846CA68B)
    v ^= v >> np.uint32(16)
    return v


def synthetic_queries(a: float, b: float, m: int, seed: int = 0) -> np.ndarray:
    """The generated query stream of pwl_eval_synthetic, as float32: x_q =
    u_q (b - a) + a with u_q = (lowbias32(q + seed) >> 8) / 2^24, a and b
    the table's float32 end knots, each operation rounded to float32."""
    q = (np.arange(m, dtype=np.uint64) + np.uint64(seed)) & np.uint64(0xFFFFFFFF)
    u = (lowbias32(q.astype(np.uint32)) >> np.uint32(8)).astype(np.float32) * np.float32(2.0 ** -24)
    a32, b32 = np.float32(a), np.float32(b)
    w = np.float32(b32 - a32)
    return (u * w + a32).astype(np.float32)


def normal_queries(desc, m: int, seed: int, sigma: float = 1.5, device="cuda", dtype=None):
    """m float32 queries normal(0, sigma) clipped to [a, b]."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.randn(m, generator=g, device=device, dtype=torch.float32)
    x.mul_(sigma).clamp_(float(desc["a"]), float(desc["b"]))
    return x if dtype is None else x.to(dtype)


def batch_functions(n_funcs: int = 4096, seed: int = 3, knots_lo: int = 16, knots_hi: int = 4096,
                    q_lo: float = 1e3, q_hi: float = 1e6):
    """Independent functions for the batched workload: kinds cycled
    (Gaussian, Lorentzian, J0); Gaussian sigma and Lorentzian gamma
    log-uniform on [0.1, 10] with domains [-4 sigma, 4 sigma] and
    [-10 gamma, 10 gamma]; J0(alpha x) with alpha uniform on [0.5, 5] on
    [0, 50]; knot counts uniform on {knots_lo..knots_hi} (intervals = knots-1);
    query counts log-uniform on [q_lo, q_hi], rounded."""
    rng = np.random.default_rng(seed)
    funcs, n_int, n_q = [], [], []
    for i in range(n_funcs):
        kind = i % 3
        if kind == 0:
            s = math.exp(rng.uniform(math.log(0.1), math.log(10.0)))
            funcs.append({"kind": "gaussian", "a": -4 * s, "b": 4 * s, "p": [1.0, 0.0, s]})
        elif kind == 1:
            g = math.exp(rng.uniform(math.log(0.1), math.log(10.0)))
            funcs.append({"kind": "lorentzian", "a": -10 * g, "b": 10 * g, "p": [1.0, 0.0, g]})
        else:
            al = rng.uniform(0.5, 5.0)
            funcs.append({"kind": "bessel_j0", "a": 0.0, "b": 50.0, "p": [1.0, al]})
        n_int.append(int(rng.integers(knots_lo, knots_hi + 1)) - 1)
        n_q.append(int(round(math.exp(rng.uniform(math.log(q_lo), math.log(q_hi))))))
    return funcs, n_int, n_q


def batch_queries(funcs, n_q, seed: int = 6, device="cuda"):
    """Concatenated float32 queries of a batch: function f's n_q[f] queries,
    uniform on its domain [a_f, b_f), follow those of functions 0..f-1.
    Returns (x, offsets) with offsets a list of F+1 ints."""
    import torch
    offsets = [0]
    for n in n_q:
        offsets.append(offsets[-1] + int(n))
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    x = torch.rand(offsets[-1], generator=g, device=device, dtype=torch.float32)
    counts = torch.tensor([int(n) for n in n_q], device=device)
    a = torch.tensor([float(f["a"]) for f in funcs], device=device, dtype=torch.float32)
    w = torch.tensor([float(f["b"] - f["a"]) for f in funcs], device=device, dtype=torch.float32)
    x.mul_(torch.repeat_interleave(w, counts, output_size=offsets[-1]))
    x.add_(torch.repeat_interleave(a, counts, output_size=offsets[-1]))
    return x, offsets


def channel_inputs(rows: int, channels: int, seed: int = 4, sigma: float = 2.0, device="cuda"):
    """x[rows, channels] float32 normal(0, sigma) for the channel-wise map."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randn(rows, channels, generator=g, device=device) * sigma


def upstream_grad(shape, seed: int = 5, device="cuda"):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randn(*shape, generator=g, device=device)
