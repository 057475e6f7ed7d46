"""Pins for the paper's error results, computed from the oracle's partitions
and values and its L2 distance:

  Result 1 / Eq. 29 : ||f - pi f||^2 on I_i = h^5/120 f''^2 exactly when f'' is
                      constant (f = x^2)
  Corollary / Result 3: best segment and P_T error^2 = h^5/720 f''^2 for f = x^2
  Result 4          : ||f - pi_{T*} f|| ~ (int |f''|^{2/5})^{5/2} / (N^2 sqrt 120)
  Result 5          : ||f - P_{T*} f|| ~ ||f - pi_{T*} f|| / sqrt 6
  Result 6          : uniform T, ||f - pi f|| ~ (b-a)^2 ||f''|| / (N^2 sqrt 120)
  O(N^-2) decay of all of them, and pi_T >= f for convex f (Section II-B).
"""
import numpy as np
import pytest

import oracle

GAUSS = {"kind": "gaussian", "a": -4.0, "b": 4.0, "p": [1.0, 0.0, 1.0]}
LOR = {"kind": "lorentzian", "a": -10.0, "b": 10.0, "p": [1.0, 0.0, 1.0]}
J0 = {"kind": "bessel_j0", "a": 0.0, "b": 50.0, "p": [1.0, 1.0]}
CONFIG = [GAUSS, LOR, J0]
SQ120 = np.sqrt(120.0)


def test_result1_equality_for_constant_second_derivative():
    # f = 3 x^2 - x: f'' = 6; (f - pi f)^2 is a quartic, so GL-16 is exact
    desc = {"kind": "poly", "a": -1.0, "b": 2.0, "p": [0.0, -1.0, 3.0]}
    rng = np.random.default_rng(0)
    k = np.concatenate([[-1.0], np.sort(rng.uniform(-1, 2, 9)), [2.0]])
    v = oracle.interp_values(desc, k)
    _, per = oracle.l2_error(desc, k, v, Q=16, per_interval=True)
    h = np.diff(k)
    assert np.allclose(per[1:], h**5 / 120.0 * 36.0, rtol=1e-12, atol=1e-18)


def test_projection_error_of_quadratic_is_one_sixth():
    # uniform partition of f = x^2: every segment of P_T is the best segment,
    # whose squared error is h^5/720 f''^2 (Corollary); pi_T has h^5/120 f''^2
    desc = {"kind": "poly", "a": 0.0, "b": 3.0, "p": [0.0, 0.0, 1.0]}
    N = 12
    k = np.linspace(0.0, 3.0, N + 1)
    h = 3.0 / N
    e_p = oracle.l2_error(desc, k, oracle.project_values(desc, k), Q=16)
    e_i = oracle.l2_error(desc, k, oracle.interp_values(desc, k), Q=16)
    assert e_p**2 == pytest.approx(N * h**5 * 4.0 / 720.0, rel=1e-12)
    assert e_i**2 == pytest.approx(N * h**5 * 4.0 / 120.0, rel=1e-12)


def _errors(desc, N):
    k = oracle.design(desc, N)
    e_i = oracle.l2_error(desc, k, oracle.interp_values(desc, k), Q=16, sub=2)
    e_p = oracle.l2_error(desc, k, oracle.project_values(desc, k), Q=16, sub=2)
    return e_i, e_p


@pytest.mark.parametrize("desc", CONFIG, ids=lambda d: d["kind"])
def test_result4_and_result5_on_optimised_partition(desc):
    GM = oracle.integral_abs_f2_pow(desc, 0.4)
    Ns = [256, 1024, 4096]
    ei, ep = zip(*[_errors(desc, N) for N in Ns])
    for N, e_i, e_p in zip(Ns, ei, ep):
        pred = GM**2.5 / (N**2 * SQ120)
        if N >= 1024:
            assert e_i / pred == pytest.approx(1.0, abs=0.05)       # Result 4
        assert e_p / e_i == pytest.approx(1 / np.sqrt(6), rel=0.05)  # Result 5
    slope = np.polyfit(np.log(Ns), np.log(ei), 1)[0]
    assert -2.05 <= slope <= -1.95


@pytest.mark.parametrize("desc", CONFIG, ids=lambda d: d["kind"])
def test_result6_uniform_partition(desc):
    f2norm = np.sqrt(oracle.integral_abs_f2_pow(desc, 2.0))
    L = desc["b"] - desc["a"]
    es = []
    Ns = [1024, 4096]
    for N in Ns:
        k = desc["a"] + np.arange(N + 1) * L / N
        e = oracle.l2_error(desc, k, oracle.interp_values(desc, k), Q=16, sub=2)
        es.append(e)
        assert e / (L**2 * f2norm / (N**2 * SQ120)) == pytest.approx(1.0, abs=0.05)
    assert np.log(es[0] / es[1]) / np.log(4) == pytest.approx(2.0, abs=0.05)


def test_optimised_partition_beats_uniform():
    # the profit of Section III-B: Result 4 / Result 6 < 1 for these functions
    for desc in CONFIG:
        N = 1024
        k = desc["a"] + np.arange(N + 1) * (desc["b"] - desc["a"]) / N
        e_u = oracle.l2_error(desc, k, oracle.interp_values(desc, k), Q=16, sub=2)
        e_o, _ = _errors(desc, N)
        assert e_o < e_u


def test_bessel_prediction_needs_resolution():
    # J0 on [0, 20]: below ~63 intervals the oscillations are under-resolved
    # and the measured error departs from Result 4; above, they agree
    desc = {"kind": "bessel_j0", "a": 0.0, "b": 20.0, "p": [1.0, 1.0]}
    GM = oracle.integral_abs_f2_pow(desc, 0.4)
    ratio = {}
    for N in (15, 255):
        e_i, _ = _errors(desc, N)
        ratio[N] = e_i / (GM**2.5 / (N**2 * SQ120))
    assert abs(ratio[255] - 1) < 0.05
    assert abs(ratio[15] - 1) > abs(ratio[255] - 1)


def test_interpolant_overestimates_convex_functions():
    for desc in ({"kind": "poly", "a": -2.0, "b": 3.0, "p": [1.0, 0.5, 2.0]},
                 {"kind": "exp", "a": -1.0, "b": 2.0, "p": [1.0, 1.5]},
                 {"kind": "lorentzian", "a": 1.0, "b": 10.0, "p": [1.0, 0.0, 1.0]}):
        k = oracle.design(desc, 33)
        x = np.linspace(desc["a"], desc["b"], 20001)
        y = oracle.evaluate(k, oracle.interp_values(desc, k), x)
        assert np.all(y >= oracle.f(desc, x) - 1e-15)
