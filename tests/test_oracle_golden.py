"""The oracle against the constants the paper prints in its error analysis
(tests/golden/paper_constants.txt).  Every check uses a function with
constant f'' (a quadratic, or a cubic for the density exponent), where the
printed relations hold with equality, so the oracle must reproduce the
constants to rounding."""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def _constants():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, value, cite = (part.strip() for part in line.split("|", 2))
            assert cite, name
            out[name] = float(value)
    return out


C = _constants()


def _quadratic(c, a, b, p0=0.3, p1=-0.7):
    # f = p0 + p1 x + (c/2) x^2: f'' = c everywhere
    return {"kind": "poly", "a": a, "b": b, "p": [p0, p1, 0.5 * c]}


def test_fixture_is_self_consistent():
    # Result 2 with eta = eta_0 = eta_1 gives Corollary 1: 1/120 - 1/144 = 1/720
    lhs = 1.0 / C["interp_sq_error_denominator"] - 1.0 / C["strict_best_segment_correction_denominator"]
    assert abs(lhs - 1.0 / C["best_segment_sq_error_denominator"]) <= 1e-15
    assert abs(C["projection_gain"] ** 2 - C["best_segment_sq_error_denominator"] / C["interp_sq_error_denominator"]) <= 1e-12
    assert C["density_exponent"] * C["bound_exponent"] == 1.0


@pytest.mark.parametrize("c,a,h", [(2.0, 0.0, 1.0), (-3.5, -1.25, 0.4), (0.8, 2.0, 3.0)])
def test_interpolant_and_best_segment_on_one_interval(c, a, h):
    desc = _quadratic(c, a, a + h)
    knots = np.array([a, a + h])
    e_pi = oracle.l2_error(desc, knots, oracle.values(desc, knots, "interp"))
    # on one interval P_T is the best line segment of Result 2
    vp = oracle.values(desc, knots, "project")
    e_p = oracle.l2_error(desc, knots, vp)
    assert abs(h ** 5 * c * c / e_pi ** 2 - C["interp_sq_error_denominator"]) <= 1e-8 * C["interp_sq_error_denominator"]
    assert abs(h ** 5 * c * c / e_p ** 2 - C["best_segment_sq_error_denominator"]) <= 1e-8 * C["best_segment_sq_error_denominator"]
    assert abs(e_pi / e_p - C["projection_gain"]) <= 1e-8
    # the minimizing offsets at both ends: (c - 2c) h^2 / 12
    dy = vp - oracle.f(desc, knots)
    want = (c - 2.0 * c) * h * h / C["delta_y_minimizer_denominator"]
    assert np.all(np.abs(dy - want) <= 1e-12 * max(1.0, abs(want)))


def test_interpolant_error_sums_over_a_nonuniform_partition():
    c = 1.7
    desc = _quadratic(c, -2.0, 3.0)
    knots = np.array([-2.0, -1.9, -1.0, 0.05, 0.5, 2.2, 3.0])
    e = oracle.l2_error(desc, knots, oracle.values(desc, knots, "interp"))
    h = np.diff(knots)
    want = math.sqrt(float(np.sum(h ** 5)) * c * c / C["interp_sq_error_denominator"])
    assert abs(e - want) <= 1e-9 * want


@pytest.mark.parametrize("N", [4, 33, 256])
def test_projection_gain_on_uniform_partition(N):
    # constant f'' on a uniform partition: the independently optimised
    # segments shift every vertex by the same -c h^2 / 12, so they join
    # continuously, P_T is their union, and the gain is exact
    c, a, b = -2.3, -1.0, 4.0
    desc = _quadratic(c, a, b)
    knots = a + (b - a) * np.arange(N + 1) / N
    e_pi = oracle.l2_error(desc, knots, oracle.values(desc, knots, "interp"))
    e_p = oracle.l2_error(desc, knots, oracle.values(desc, knots, "project"))
    assert abs(e_pi / e_p - C["projection_gain"]) <= 1e-8


def test_bound_exponent_on_the_designed_partition():
    # f'' constant: the designed partition is uniform and Result 4 holds
    # with equality, with the density integral G_M of the design itself
    c, a, b = 2.0, -1.0, 2.0
    desc = _quadratic(c, a, b)
    for N in (3, 50, 700):
        knots, aux = oracle.design(desc, N, return_aux=True)
        e = oracle.l2_error(desc, knots, oracle.values(desc, knots, "interp"))
        g = aux["G"][-1]
        assert abs(g - abs(c) ** C["density_exponent"] * (b - a)) <= 1e-12 * g
        want = g ** C["bound_exponent"] / (N * N * math.sqrt(C["interp_sq_error_denominator"]))
        assert abs(e - want) <= 1e-9 * want


def test_density_exponent_gives_the_cubic_power_law():
    # f = x^3 on [0, 1]: |f''| = 6x, so F(x) is proportional to
    # x^{1 + density_exponent} and x_i = (i / N)^{1 / (1 + density_exponent)}
    desc = {"kind": "poly", "a": 0.0, "b": 1.0, "p": [0.0, 0.0, 0.0, 1.0]}
    N = 40
    knots = oracle.design(desc, N, 1 << 18)
    want = (np.arange(N + 1) / N) ** (1.0 / (1.0 + C["density_exponent"]))
    assert np.abs(knots - want).max() <= 2e-6
