"""Pins for the oracle's design step: local knot density (Eq. 16), cumulative
distribution F (Eq. 18) and the knots F(x_i) = i/N (Eq. 17).

Closed forms:
  f = x^2      : |f''| constant, F linear          -> uniform knots
  f = x^3 [0,1]: |f''|^{2/5} ~ x^{2/5}, F = x^{7/5}  -> x_i = (i/N)^{5/7}
  f = e^x      : F ~ e^{2x/5} - e^{2a/5}            -> x_i = 5/2 ln(e^{2a/5} + i/N (e^{2b/5} - e^{2a/5}))
The integral of |f''|^{2/5} is checked against scipy's adaptive quadrature of
an independently written f'' (J0'' from the J2 recurrence).
"""
import numpy as np
import pytest

import oracle

def test_quadratic_gives_uniform_knots():
    for (a, b, N) in [(0.0, 1.0, 7), (-3.0, 5.0, 64), (-4.0, 4.0, 1024)]:
        desc = {"kind": "poly", "a": a, "b": b, "p": [0.3, -1.0, 2.5]}
        k = oracle.design(desc, N)
        ref = a + np.arange(N + 1) * (b - a) / N
        assert np.abs(k - ref).max() <= 1e-13 * (b - a)


def test_cubic_knots_follow_power_law_and_converge_in_M():
    desc = {"kind": "poly", "a": 0.0, "b": 1.0, "p": [0.0, 0.0, 0.0, 1.0]}
    N = 16
    ref = (np.arange(N + 1) / N) ** (5.0 / 7.0)
    errs = []
    for M in [2**12, 2**14, 2**16]:
        k = oracle.design(desc, N, M)
        errs.append(np.abs(k - ref).max())
    assert errs[-1] < 1e-5
    # the midpoint rule on x^{2/5} has error O(M^{-7/5}) near 0: rate ~ 4^{1.4} = 7 per step
    assert errs[0] / errs[1] > 5 and errs[1] / errs[2] > 5


def test_exponential_closed_form_knots():
    a, b, N = -1.0, 2.0, 37
    desc = {"kind": "exp", "a": a, "b": b, "p": [2.0, 1.0]}
    i = np.arange(N + 1) / N
    ref = 2.5 * np.log(np.exp(0.4 * a) + i * (np.exp(0.4 * b) - np.exp(0.4 * a)))
    k = oracle.design(desc, N, 64 * N)
    assert np.abs(k - ref).max() < 1e-6
    k2 = oracle.design(desc, N, 4 * 64 * N)
    assert np.abs(k2 - ref).max() < np.abs(k - ref).max() / 10  # O(delta^2)


def _scipy_f2(desc, x):
    sc = pytest.importorskip("scipy.special")
    p = desc["p"]
    if desc["kind"] == "gaussian":
        u = (x - p[1]) / p[2]
        return p[0] * (u * u - 1) / p[2] ** 2 * np.exp(-u * u / 2)
    if desc["kind"] == "lorentzian":
        u = (x - p[1]) / p[2]
        return p[0] * (6 * u * u - 2) / (p[2] ** 2 * (1 + u * u) ** 3)
    if desc["kind"] == "bessel_j0":
        z = p[1] * x
        # J0'' = (J2 - J0) / 2 (recurrence), independent of the J1/z form
        return p[0] * p[1] ** 2 * 0.5 * (sc.jv(2, z) - sc.j0(z))


CONFIG_FUNCS = [
    {"kind": "gaussian", "a": -4.0, "b": 4.0, "p": [1.0, 0.0, 1.0]},
    {"kind": "lorentzian", "a": -10.0, "b": 10.0, "p": [1.0, 0.0, 1.0]},
    {"kind": "bessel_j0", "a": 0.0, "b": 50.0, "p": [1.0, 1.0]},
]


@pytest.mark.parametrize("desc", CONFIG_FUNCS, ids=lambda d: d["kind"])
def test_density_integral_matches_adaptive_quadrature(desc):
    integrate = pytest.importorskip("scipy.integrate")
    ref, _ = integrate.quad(lambda t: abs(_scipy_f2(desc, t)) ** 0.4, desc["a"], desc["b"],
                            limit=2000, epsabs=1e-13, epsrel=1e-13)
    # midpoint rule; the cusps of |f''|^{2/5} at zeros of f'' limit it to O(M^{-7/5})
    for N, tol in [(256, 1e-5), (1024, 2e-6)]:
        _, aux = oracle.design(desc, N, 64 * N, return_aux=True)
        assert aux["G"][-1] == pytest.approx(ref, rel=tol)


@pytest.mark.parametrize("desc", CONFIG_FUNCS, ids=lambda d: d["kind"])
def test_knots_equidistribute_independent_cdf(desc):
    # F(x_i) = i/N (Eq. 17) with F from scipy's quadrature, not from the oracle
    integrate = pytest.importorskip("scipy.integrate")
    N = 32
    dens = lambda t: abs(_scipy_f2(desc, t)) ** 0.4
    for M, tol in [(64 * N, 1e-4), (2**16, 2e-6)]:
        k = oracle.design(desc, N, M)
        assert np.all(np.diff(k) > 0)
        pieces = np.array([integrate.quad(dens, k[j], k[j + 1], limit=500, epsabs=1e-12)[0]
                           for j in range(N)])
        # every interval carries 1/N of the mass of |f''|^{2/5}, up to the
        # midpoint-rule discretisation of F
        assert np.abs(pieces / pieces.sum() - 1.0 / N).max() < tol


# Hand-derived inversions (delta = 1 in every case).  G_k = sum_{j<k} d_j;
# tau_i = i G_M / N; cell = largest k with G_k <= tau and d_k > 0;
# x_i = a + k + (tau - G_k) / d_k.
#  A: d = [1,0,0,1], N=2: G=[0,1,1,1,2]; tau=1 -> k=3 (G_3=1)  -> x=3
#  B: d = [2,0,1,1], N=4: G=[0,2,2,3,4]; tau=1 -> k=0 -> 0.5; tau=2 -> k=2 -> 2;
#     tau=3 -> k=3 -> 3
#  C: d = [1,1,0,0], N=2: G=[0,1,2,2,2]; tau=1 -> k=1 -> 1
#  D: d = [0,0,3,1], a=-1, N=4: G=[0,0,0,3,4]; tau=1 -> k=2 -> -1+2+1/3;
#     tau=2 -> -1+2+2/3; tau=3 -> k=3 -> 2
INVERSION_CASES = [
    ([1, 0, 0, 1], 0.0, 4.0, 2, [0, 3, 4]),
    ([2, 0, 1, 1], 0.0, 4.0, 4, [0, 0.5, 2, 3, 4]),
    ([1, 1, 0, 0], 0.0, 4.0, 2, [0, 1, 4]),
    ([0, 0, 3, 1], -1.0, 3.0, 4, [-1, 4.0 / 3.0, 5.0 / 3.0, 2, 3]),
]


@pytest.mark.parametrize("case", INVERSION_CASES)
def test_inversion_skips_zero_density_runs(case):
    d, a, b, N, expect = case
    d = np.array(d, dtype=np.float64)
    G = oracle.cumulative(d, (b - a) / d.size)
    k, rc = oracle.invert(d, G, a, b, N)
    assert rc == 0
    assert np.allclose(k, expect, rtol=0, atol=1e-15), k


def test_linear_function_falls_back_to_uniform():
    desc = {"kind": "poly", "a": -2.0, "b": 3.0, "p": [1.0, 4.0]}
    k, aux = oracle.design(desc, 10, 640, return_aux=True)
    assert aux["rc"] == 1
    assert np.allclose(k, -2.0 + np.arange(11) * 0.5, atol=1e-15)


def test_cumulative_is_compensated_sum():
    rng = np.random.default_rng(0)
    d = rng.random(100000) * 1e3
    d[::7] = 1e-9
    G = oracle.cumulative(d, 0.25)
    import math
    ref = [0.0]
    for j in range(1, d.size + 1, 9973):
        ref_j = 0.25 * math.fsum(d[:j])
        assert abs(G[j] - ref_j) <= 4e-16 * abs(ref_j)
