"""Pins for the oracle's test functions f and f'' (Sections V-VI).

f is checked against numpy/scipy library routines and f'' against symbolic
differentiation (sympy) and central second differences of f, so a dropped
term or wrong sign in either formula fails here.
"""
import numpy as np
import pytest

import oracle

FUNCS = [
    {"kind": "gaussian", "a": -4.0, "b": 4.0, "p": [1.0, 0.0, 1.0]},
    {"kind": "gaussian", "a": -3.0, "b": 5.0, "p": [0.7, 0.4, 1.7]},
    {"kind": "lorentzian", "a": -10.0, "b": 10.0, "p": [1.0, 0.0, 1.0]},
    {"kind": "lorentzian", "a": -2.0, "b": 6.0, "p": [1.0 / np.pi, 0.5, 0.3]},
    {"kind": "bessel_j0", "a": 0.0, "b": 50.0, "p": [1.0, 1.0]},
    {"kind": "bessel_j0", "a": -3.0, "b": 20.0, "p": [0.5, 2.3]},
    {"kind": "poly", "a": -4.0, "b": 3.0, "p": [24.0, -2.0, -23.0, 1.0, 3.0, 1.0]},
    {"kind": "exp", "a": -1.0, "b": 2.0, "p": [1.5, 1.3]},
]


def _sym(desc):
    sp = pytest.importorskip("sympy")
    x = sp.symbols("x")
    p = [sp.Float(v, 30) for v in desc["p"]]
    k = desc["kind"]
    if k == "gaussian":
        e = p[0] * sp.exp(-((x - p[1]) ** 2) / (2 * p[2] ** 2))
    elif k == "lorentzian":
        e = p[0] / (1 + ((x - p[1]) / p[2]) ** 2)
    elif k == "bessel_j0":
        e = p[0] * sp.besselj(0, p[1] * x)
    elif k == "poly":
        e = sum(c * x ** i for i, c in enumerate(p))
    elif k == "exp":
        e = p[0] * sp.exp(p[1] * x)
    return sp, x, e


def _lib_f(desc, x):
    sc = pytest.importorskip("scipy.special")
    p = desc["p"]
    k = desc["kind"]
    if k == "gaussian":
        return p[0] * np.exp(-((x - p[1]) ** 2) / (2 * p[2] ** 2))
    if k == "lorentzian":
        return p[0] / (1 + ((x - p[1]) / p[2]) ** 2)
    if k == "bessel_j0":
        return p[0] * sc.j0(p[1] * x)
    if k == "poly":
        return np.polynomial.polynomial.polyval(x, p)
    if k == "exp":
        return p[0] * np.exp(p[1] * x)


@pytest.mark.parametrize("desc", FUNCS, ids=lambda d: d["kind"])
def test_f_matches_library(desc):
    x = np.linspace(desc["a"], desc["b"], 257)
    got = oracle.f(desc, x)
    ref = _lib_f(desc, x)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-14 * scale


@pytest.mark.parametrize("desc", FUNCS, ids=lambda d: d["kind"])
def test_f2_matches_symbolic_second_derivative(desc):
    sp, x, e = _sym(desc)
    d2 = sp.diff(e, x, 2)
    xs = np.linspace(desc["a"], desc["b"], 97)
    xs = xs[np.abs(xs) > 1e-3]  # sympy's besselj derivative form is singular at 0
    ref = np.array([float(d2.subs(x, sp.Float(v, 30)).evalf(25)) for v in xs])
    got = oracle.f2(desc, xs)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-13 * scale


@pytest.mark.parametrize("desc", FUNCS, ids=lambda d: d["kind"])
def test_f2_matches_second_difference_of_f(desc):
    # central second difference of the oracle's own f: independent of f''
    h = 1e-3 * (desc["b"] - desc["a"]) / 8
    xs = np.linspace(desc["a"] + 2 * h, desc["b"] - 2 * h, 61)
    fd = (oracle.f(desc, xs + h) - 2 * oracle.f(desc, xs) + oracle.f(desc, xs - h)) / h**2
    got = oracle.f2(desc, xs)
    scale = np.abs(got).max()
    assert np.abs(got - fd).max() <= 2e-5 * scale


def test_j0_second_derivative_at_origin():
    # J0''(0) = -1/2, so (A J0(alpha x))'' = -A alpha^2 / 2 at x = 0
    desc = {"kind": "bessel_j0", "a": 0.0, "b": 1.0, "p": [1.3, 2.0]}
    assert oracle.f2(desc, [0.0])[0] == pytest.approx(-1.3 * 4.0 / 2.0, rel=1e-15)
    assert oracle.f2(desc, [1e-9])[0] == pytest.approx(-1.3 * 4.0 / 2.0, rel=1e-12)


@pytest.mark.parametrize("desc", FUNCS[:6], ids=lambda d: d["kind"])
def test_f_many_matches_library(desc):
    x = np.linspace(desc["a"], desc["b"], 1001)
    assert np.allclose(oracle.f_many(desc, x), _lib_f(desc, x), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("A,alpha", [(1.0, 1.0), (2.0, 0.5), (0.3, 3.7)])
def test_j0_one_term_is_the_leading_term_of_hankels_expansion(A, alpha):
    # J0(z) = sqrt(2/(pi z)) [cos w (1 - 9/(128 z^2) + ...) + sin w / (8 z) - ...],
    # w = z - pi/4 (DLMF 10.17.3 with a_1(0) = -1/8, a_2(0) = 9/128,
    # a_3(0) = -225/3072); for real z > 0 the remainder after a term is
    # bounded by the next term (DLMF 10.17(iii)).  So J0 minus the oracle's
    # one-term form, minus the 1/(8z) sine term, is within the 9/(128 z^2)
    # and 225/(3072 z^3) terms: a wrong phase, sign or amplitude fails.
    sc = pytest.importorskip("scipy.special")
    desc = {"kind": "bessel_j0", "a": 0.0, "b": 100.0, "p": [A, alpha]}
    z = np.linspace(8.0, 400.0, 20001)
    x = z / alpha
    s = np.sqrt(2.0 / (np.pi * z))
    w = z - np.pi / 4
    one = oracle.j0_one_term(desc, x)
    rest = A * sc.j0(z) - one - A * s * np.sin(w) / (8 * z)
    # (+ the rounding of z = alpha (z / alpha) inside the oracle: ~ulp(z))
    bound = A * s * (9.0 / (128 * z**2) + 225.0 / (3072 * z**3)) + 4e-16 * A * z
    assert np.all(np.abs(rest) <= bound)
    # and the one-term form is not J0 itself: its error is the 1/(8z) term
    err = np.abs(A * sc.j0(z) - one)
    assert np.max(err / (A * s / (8 * z))) > 0.9
