"""Pins for the oracle's CPWL evaluation (Algorithm 1) and its gradients.

Evaluation is checked against numpy's np.interp (same clamping semantics), a
brute-force linear scan written out in Python, and exactness on linear
functions.  Gradients are checked against central finite differences in FP64
and the invariants sum_k dy/dv_k = 1 and dy/dx + sum_k dy/dx_k = 0.
"""
import numpy as np
import pytest

import oracle


def _knots(rng, a, b, N):
    h = (b - a) / N
    k = a + h * (np.arange(N + 1) + rng.uniform(-0.4, 0.4, N + 1))
    k[0], k[-1] = a, b
    return k


def test_matches_numpy_interp():
    rng = np.random.default_rng(0)
    for N in (1, 2, 3, 17, 1000):
        k = _knots(rng, -2.0, 5.0, N)
        v = rng.normal(size=N + 1)
        x = rng.uniform(-3.0, 6.0, 5000)
        x[:N + 1] = k  # exactly at the knots
        y = oracle.evaluate(k, v, x)
        ref = np.interp(x, k, v)
        assert np.abs(y - ref).max() <= 4e-16 * np.abs(v).max() * 4


def test_matches_brute_force_scan():
    rng = np.random.default_rng(1)
    N = 9
    k = _knots(rng, 0.0, 1.0, N)
    v = rng.normal(size=N + 1)
    xs = list(rng.uniform(-0.2, 1.2, 300)) + list(k) + [0.0, 1.0]
    y = oracle.evaluate(k, v, xs)
    for x, got in zip(xs, y):
        xc = min(max(x, k[0]), k[-1])
        i = 1
        while i < N and not (k[i - 1] <= xc < k[i]):
            i += 1
        d = (xc - k[i - 1]) / (k[i] - k[i - 1])
        assert got == pytest.approx((1 - d) * v[i - 1] + d * v[i], abs=1e-15)


def test_edge_cases():
    k = np.array([-1.0, 0.0, 2.0, 3.0])
    v = np.array([1.0, -1.0, 3.0, 0.5])
    x = np.array([-5.0, -1.0, 0.0, 2.0, 3.0, 7.0, np.nan, 1.0, 2.5])
    y = oracle.evaluate(k, v, x)
    assert np.array_equal(y[:6], [1.0, 1.0, -1.0, 3.0, 0.5, 0.5])
    assert np.isnan(y[6])
    assert y[7] == 1.0 and y[8] == 1.75
    assert oracle.evaluate(k, v, np.zeros(0)).size == 0


def test_linear_function_is_exact():
    rng = np.random.default_rng(2)
    k = _knots(rng, -1.0, 1.0, 50)
    v = 3.0 * k - 0.25
    x = rng.uniform(-1, 1, 2000)
    assert np.abs(oracle.evaluate(k, v, x) - (3.0 * x - 0.25)).max() < 1e-15


def _y(k, v, x):
    return oracle.evaluate(k, v, np.array([x]))[0]


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    N = 6
    k = _knots(rng, -1.0, 2.0, N)
    v = rng.normal(size=N + 1)
    xs = rng.uniform(-1.0, 2.0, 40)
    # keep queries away from knots (one-sided derivatives there)
    xs = xs[np.min(np.abs(xs[:, None] - k[None, :]), axis=1) > 1e-3]
    gy = rng.normal(size=xs.size)
    gx, gv, gxk, _, _ = oracle.evaluate_grad(k, v, xs, gy)
    eps = 1e-6
    fd_gx = np.array([(_y(k, v, x + eps) - _y(k, v, x - eps)) / (2 * eps) for x in xs]) * gy
    assert np.abs(gx - fd_gx).max() < 1e-7 * np.abs(gx).max()
    for j in range(N + 1):
        e = np.zeros(N + 1)
        e[j] = eps
        fv = sum(g * (_y(k, v + e, x) - _y(k, v - e, x)) / (2 * eps) for x, g in zip(xs, gy))
        assert abs(gv[j] - fv) < 1e-7 * max(1.0, abs(gv).max())
        fk = sum(g * (_y(k + e, v, x) - _y(k - e, v, x)) / (2 * eps) for x, g in zip(xs, gy))
        assert abs(gxk[j] - fk) < 1e-6 * max(1.0, abs(gxk).max())


def test_gradient_invariants():
    rng = np.random.default_rng(4)
    N = 40
    k = _knots(rng, 0.0, 10.0, N)
    v = rng.normal(size=N + 1)
    x = rng.uniform(0.0, 10.0, 1)
    for xq in list(x) + [3.3, 7.0]:
        gx, gv, gxk, _, _ = oracle.evaluate_grad(k, v, [xq], [1.0])
        # y is an affine combination of the v_k: sum dy/dv_k = 1
        assert abs(gv.sum() - 1.0) < 1e-15
        # shifting x and every knot together leaves y unchanged
        assert abs(gx[0] + gxk.sum()) < 1e-13


def test_gradient_of_clamped_and_nan_queries():
    k = np.array([0.0, 1.0, 2.0])
    v = np.array([1.0, 3.0, 2.0])
    gx, gv, gxk, _, _ = oracle.evaluate_grad(k, v, [-1.0, 5.0, np.nan], [2.0, 3.0, 7.0])
    assert gx[0] == 0.0 and gx[1] == 0.0 and np.isnan(gx[2])
    assert np.array_equal(gv, [2.0, 0.0, 3.0])
    assert np.array_equal(gxk, [0.0, 0.0, 0.0])
