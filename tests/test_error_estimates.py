"""A priori errors and the N for a target error (Results 4-6, Section III-B):
the host formulas (no GPU) pinned to closed forms and to the oracle's L2
errors, and the GPU integrals behind them against the oracle."""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pwl():
    import paper_1510_02975_gb300 as m
    from paper_1510_02975_gb300 import _build
    _build.build()
    return m


def test_quadratic_prediction_is_the_exact_error(pwl):
    # f = x^2: f'' = 2, so int |f''|^{2/5} = 2^{2/5} (b - a) and ||f''||^2 =
    # 4 (b - a); T* is uniform and the interpolant's error on it is exactly
    # 2 (b - a)^{5/2} / (N^2 sqrt(120)) for every N (Result 1 holds with equality)
    a, b = -1.0, 2.0
    i25, isq = 2.0 ** 0.4 * (b - a), 4.0 * (b - a)
    desc = {"kind": "poly", "a": a, "b": b, "p": [0.0, 0.0, 1.0]}
    for N in (1, 7, 64, 1000):
        exact = 2.0 * (b - a) ** 2.5 / (N * N * math.sqrt(120.0))
        for uniform in (False, True):
            got = pwl.pwl_predicted_error(i25, isq, a, b, N, "interp", uniform)
            assert abs(got - exact) <= 1e-14 * exact
        knots = a + (b - a) * np.arange(N + 1) / N
        e = oracle.l2_error(desc, knots, oracle.values(desc, knots, "interp"))
        assert abs(e - exact) <= 1e-9 * exact


def test_projection_gains_sqrt6_and_n_is_minimal(pwl):
    i25, isq, a, b = 3.7, 11.0, 0.0, 5.0
    for uniform in (False, True):
        for N in (3, 100, 4096):
            pi = pwl.pwl_predicted_error(i25, isq, a, b, N, "interp", uniform)
            pt = pwl.pwl_predicted_error(i25, isq, a, b, N, "project", uniform)
            assert abs(pi / pt - math.sqrt(6.0)) <= 1e-14
        for target in (1e-3, 1e-6, 3.3e-9):
            for form in ("interp", "project"):
                n = pwl.pwl_n_for_error(i25, isq, a, b, target, form, uniform)
                assert pwl.pwl_predicted_error(i25, isq, a, b, n, form, uniform) <= target
                if n > 1:
                    assert pwl.pwl_predicted_error(i25, isq, a, b, n - 1, form, uniform) > target
    # f linear: no error at any N
    assert pwl.pwl_n_for_error(0.0, 0.0, 0.0, 1.0, 1e-12) == 1


def test_error_arguments_are_rejected(pwl):
    from paper_1510_02975_gb300 import PwlError
    with pytest.raises(PwlError):
        pwl.pwl_predicted_error(-1.0, 1.0, 0.0, 1.0, 10)
    with pytest.raises(PwlError):
        pwl.pwl_predicted_error(1.0, 1.0, 1.0, 0.0, 10)
    with pytest.raises(PwlError):
        pwl.pwl_predicted_error(1.0, 1.0, 0.0, 1.0, 0)
    with pytest.raises(PwlError):
        pwl.pwl_n_for_error(1.0, 1.0, 0.0, 1.0, 0.0)
    with pytest.raises(PwlError):
        pwl.pwl_n_for_error(1e6, 1.0, 0.0, 1.0, 1e-30)  # beyond the largest N


@pytest.mark.parametrize("name,a,b,p", [("gaussian", -4.0, 4.0, [1.0, 0.0, 1.0]),
                                        ("lorentzian", -10.0, 10.0, [1.0, 0.0, 1.0])])
def test_prediction_matches_oracle_error_on_optimised_partition(pwl, name, a, b, p):
    # Result 4 (interpolant) and Result 5 (projection) at N = 2048, with the
    # integral of |f''|^{2/5} from the oracle's quadrature: within 5%
    desc = {"kind": name, "a": a, "b": b, "p": p}
    i25 = oracle.integral_abs_f2_pow(desc, 0.4)
    isq = oracle.integral_abs_f2_pow(desc, 2.0)
    N = 2048
    knots = oracle.design(desc, N)
    for form in ("interp", "project"):
        e = oracle.l2_error(desc, knots, oracle.values(desc, knots, form))
        pred = pwl.pwl_predicted_error(i25, isq, a, b, N, form)
        assert abs(pred / e - 1.0) <= 0.05, (form, pred, e)
    # Result 6 on the uniform partition
    ku = a + (b - a) * np.arange(N + 1) / N
    eu = oracle.l2_error(desc, ku, oracle.values(desc, ku, "interp"))
    assert abs(pwl.pwl_predicted_error(i25, isq, a, b, N, "interp", True) / eu - 1.0) <= 0.05


@pytest.mark.gpu
@pytest.mark.parametrize("desc", [
    {"kind": "gaussian", "a": -4.0, "b": 4.0, "p": [1.0, 0.0, 1.0]},
    {"kind": "lorentzian", "a": -10.0, "b": 10.0, "p": [1.0, 0.0, 1.0]},
    {"kind": "bessel_j0", "a": 0.0, "b": 50.0, "p": [1.0, 3.0]},
    # f'' = 9 e^{3 x} spans 3e-10 .. 2e11: the GPU's |f''|^{2/5} (an
    # inverse-fifth-root iteration) against the oracle's C library pow (the
    # midpoint rule on f''^2 stays within 6e-9 of the quadrature here)
    {"kind": "exp", "a": -8.0, "b": 8.0, "p": [1.0, 3.0]},
])
def test_error_constants_match_oracle(pwl, desc):
    M = 1 << 18
    out = pwl.pwl_error_constants(desc, M).cpu().numpy()
    # the same midpoint rule as the design: G_M of the oracle's design
    _, aux = oracle.design(desc, 64, M, return_aux=True)
    assert abs(out[0] - aux["G"][-1]) <= 1e-12 * aux["G"][-1]
    # the integral of f''^2 against the oracle's Gauss-Legendre quadrature
    ref = oracle.integral_abs_f2_pow(desc, 2.0)
    assert abs(out[1] - ref) <= 1e-8 * ref


@pytest.mark.gpu
def test_error_constants_closed_forms(pwl):
    # f = A e^{lam x}: f'' = A lam^2 e^{lam x}
    A, lam, a, b = 1.5, 0.7, -2.0, 3.0
    desc = {"kind": "exp", "a": a, "b": b, "p": [A, lam]}
    out = pwl.pwl_error_constants(desc, 1 << 20).cpu().numpy()
    c = A * lam * lam
    i25 = c ** 0.4 * (math.exp(0.4 * lam * b) - math.exp(0.4 * lam * a)) / (0.4 * lam)
    isq = c * c * (math.exp(2 * lam * b) - math.exp(2 * lam * a)) / (2 * lam)
    # midpoint rule: relative error ~ (delta^2 / 24) (rate)^2
    assert abs(out[0] - i25) <= 1e-9 * i25
    assert abs(out[1] - isq) <= 1e-9 * isq
    # f = x^2: constant f'' is integrated exactly
    q = {"kind": "poly", "a": -1.0, "b": 2.0, "p": [0.0, 0.0, 1.0]}
    out = pwl.pwl_error_constants(q, 1000).cpu().numpy()
    assert abs(out[0] - 2.0 ** 0.4 * 3.0) <= 1e-13 and abs(out[1] - 12.0) <= 1e-12
