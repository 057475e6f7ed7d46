"""Pins for the oracle's vertex values: interpolant pi_T (Eq. 3) and L2
projection P_T (Eqs. 4-6: Gram system, load vector, Thomas algorithm).

Independent references: numpy's Gauss-Legendre rule and dense solver, scipy's
adaptive quadrature of hat-weighted integrands built with np.interp, dense
least squares on a fine grid, and the closed form c_i = x_i^2 - h^2/6 for
f = x^2 on a uniform partition (independently optimised segments shift both
ends by -h^2/12 * (2 - 1) - ... = -h^2/6, which is continuous, hence P_T).
"""
import numpy as np
import pytest

import oracle

GAUSS = {"kind": "gaussian", "a": -4.0, "b": 4.0, "p": [1.0, 0.0, 1.0]}
LOR = {"kind": "lorentzian", "a": -10.0, "b": 10.0, "p": [1.0, 0.0, 1.0]}
J0 = {"kind": "bessel_j0", "a": 0.0, "b": 50.0, "p": [1.0, 1.0]}


def _random_knots(rng, a, b, N):
    # jittered uniform knots: every interval is at least 0.2 (b - a) / N long,
    # so quadrature-node rounding (~eps |x| / h) stays far below the tolerances
    h = (b - a) / N
    k = a + h * (np.arange(N + 1) + rng.uniform(-0.4, 0.4, N + 1))
    k[0], k[-1] = a, b
    return k


@pytest.mark.parametrize("Q", [1, 2, 3, 5, 8, 16, 20])
def test_gauss_legendre_matches_numpy(Q):
    x, w = oracle.gauss_legendre(Q)
    xr, wr = np.polynomial.legendre.leggauss(Q)
    assert np.abs(x - xr).max() < 1e-14
    assert np.abs(w - wr).max() < 1e-14
    # exact for polynomials of degree <= 2Q - 1
    for k in range(2 * Q):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x**k) - exact) < 1e-13


def test_interpolant_is_exact_at_knots():
    rng = np.random.default_rng(1)
    for desc in (GAUSS, LOR, J0):
        k = _random_knots(rng, desc["a"], desc["b"], 50)
        v = oracle.interp_values(desc, k)
        assert np.array_equal(v, oracle.f(desc, k))
        assert np.array_equal(oracle.evaluate(k, v, k), v)


def test_gram_matches_quadrature_of_hat_products():
    rng = np.random.default_rng(2)
    k = _random_knots(rng, -1.0, 2.0, 9)
    lo, di, up = oracle.gram(k)
    n = k.size
    # hats from np.interp of unit vectors; integrate products exactly with
    # numpy's 4-point rule on every interval (products are quadratic there)
    xg, wg = np.polynomial.legendre.leggauss(4)
    M = np.zeros((n, n))
    eye = np.eye(n)
    for j in range(1, n):
        t = 0.5 * (k[j - 1] + k[j]) + 0.5 * (k[j] - k[j - 1]) * xg
        w = 0.5 * (k[j] - k[j - 1]) * wg
        phis = np.array([np.interp(t, k, eye[i]) for i in range(n)])
        M += (phis * w) @ phis.T
    assert np.allclose(np.diag(M), di, rtol=1e-14, atol=0)
    assert np.allclose(np.diag(M, 1), up[:-1], rtol=1e-14, atol=0)
    assert np.allclose(np.diag(M, -1), lo[1:], rtol=1e-14, atol=0)
    assert np.abs(M - np.diag(np.diag(M)) - np.diag(np.diag(M, 1), 1)
                  - np.diag(np.diag(M, -1), -1)).max() == 0.0
    # strictly diagonally dominant (Section II-B)
    assert np.all(di > np.abs(lo) + np.abs(up))


@pytest.mark.parametrize("desc", [GAUSS, LOR, J0], ids=lambda d: d["kind"])
def test_load_vector_matches_adaptive_quadrature(desc):
    integrate = pytest.importorskip("scipy.integrate")
    rng = np.random.default_rng(3)
    k = _random_knots(rng, desc["a"], desc["b"], 12)
    b = oracle.load_vector(desc, k, Q=16)
    eye = np.eye(k.size)
    fx = lambda t: float(oracle.f(desc, [t])[0])
    for i in range(k.size):
        lo_, hi_ = k[max(i - 1, 0)], k[min(i + 1, k.size - 1)]
        ref = integrate.quad(lambda t: fx(t) * np.interp(t, k, eye[i]), lo_, hi_,
                             points=[k[i]], limit=200, epsabs=1e-14, epsrel=1e-12)[0]
        assert abs(b[i] - ref) <= 1e-9 * max(1.0, abs(ref))


def test_thomas_matches_dense_solve():
    rng = np.random.default_rng(4)
    n = 200
    lo = rng.uniform(-1, 1, n)
    up = rng.uniform(-1, 1, n)
    di = np.abs(lo) + np.abs(up) + rng.uniform(0.5, 2, n)
    rhs = rng.normal(size=n)
    x = oracle.thomas(lo, di, up, rhs)
    A = np.diag(di) + np.diag(up[:-1], 1) + np.diag(lo[1:], -1)
    ref = np.linalg.solve(A, rhs)
    assert np.abs(x - ref).max() < 1e-13 * np.abs(ref).max()
    # size 1 and 2 edge cases
    assert oracle.thomas([0.0], [4.0], [0.0], [2.0])[0] == 0.5
    x2 = oracle.thomas([0.0, 1.0], [3.0, 3.0], [1.0, 0.0], [4.0, 5.0])
    assert np.allclose(x2, np.linalg.solve([[3.0, 1.0], [1.0, 3.0]], [4.0, 5.0]), atol=1e-15)


def test_projection_reproduces_linear_functions():
    rng = np.random.default_rng(5)
    for N in (1, 2, 7, 100):
        k = _random_knots(rng, -3.0, 4.0, N)
        desc = {"kind": "poly", "a": -3.0, "b": 4.0, "p": [0.7, -1.9]}
        c = oracle.project_values(desc, k)
        ref = 0.7 - 1.9 * k
        assert np.abs(c - ref).max() < 5e-14 * np.abs(ref).max()


@pytest.mark.parametrize("N", [1, 2, 5, 64])
def test_projection_of_quadratic_on_uniform_partition(N):
    # closed form from the optimal end offsets of Result 2's proof with
    # f'' = 2 constant: both ends move by (2 - 4) h^2 / 12 = -h^2 / 6
    a, b = -1.0, 2.0
    k = a + np.arange(N + 1) * (b - a) / N
    h = (b - a) / N
    desc = {"kind": "poly", "a": a, "b": b, "p": [0.0, 0.0, 1.0]}
    c = oracle.project_values(desc, k)
    assert np.abs(c - (k**2 - h * h / 6.0)).max() < 1e-13


@pytest.mark.parametrize("desc,N", [(GAUSS, 3), (LOR, 5), (J0, 8),
                                    ({"kind": "poly", "a": -4.0, "b": 3.0,
                                      "p": [24.0, -2.0, -23.0, 1.0, 3.0, 1.0]}, 6)],
                         ids=["gauss", "lorentz", "j0", "quintic"])
def test_projection_matches_dense_least_squares(desc, N):
    # brute force: minimise sum (f(t) - sum c_i phi_i(t))^2 over a fine
    # uniform grid (trapezoid weights) with numpy's least-squares solver
    rng = np.random.default_rng(6)
    k = _random_knots(rng, desc["a"], desc["b"], N)
    t = np.linspace(desc["a"], desc["b"], 200001)
    w = np.full(t.size, t[1] - t[0])
    w[0] = w[-1] = 0.5 * (t[1] - t[0])
    eye = np.eye(N + 1)
    Phi = np.stack([np.interp(t, k, eye[i]) for i in range(N + 1)], axis=1)
    sw = np.sqrt(w)
    ref = np.linalg.lstsq(Phi * sw[:, None], oracle.f(desc, t) * sw, rcond=None)[0]
    c = oracle.project_values(desc, k, Q=16)
    scale = np.abs(oracle.f(desc, t)).max()
    # grid discretisation error of the trapezoid rule ~ (dt)^2
    assert np.abs(c - ref).max() < 2e-6 * scale


# quad may report that it cannot certify its 1e-14 absolute tolerance on the
# J0 products; the assertion below bounds the integral itself
@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("desc", [GAUSS, LOR, J0], ids=lambda d: d["kind"])
def test_projection_residual_is_orthogonal(desc):
    # <f - P_T f, phi_j> = 0 (Eq. 5), the integral by scipy's quadrature
    integrate = pytest.importorskip("scipy.integrate")
    rng = np.random.default_rng(7)
    k = _random_knots(rng, desc["a"], desc["b"], 10)
    # wide intervals (N = 10): Q = 32 resolves f to rounding on each of them
    c = oracle.project_values(desc, k, Q=32)
    eye = np.eye(k.size)
    fx = lambda t: float(oracle.f(desc, [t])[0])
    for j in range(k.size):
        lo_, hi_ = k[max(j - 1, 0)], k[min(j + 1, k.size - 1)]
        r = integrate.quad(lambda t: (fx(t) - np.interp(t, k, c)) * np.interp(t, k, eye[j]),
                           lo_, hi_, points=[k[j]], limit=200, epsabs=1e-14)[0]
        assert abs(r) < 1e-13


@pytest.mark.parametrize("desc", [GAUSS, LOR, J0], ids=lambda d: d["kind"])
def test_projection_is_no_worse_than_interpolant(desc):
    # Eq. 7: P_T f is the best L2 approximation in the CPWL space
    for N in (8, 64, 512):
        k = oracle.design(desc, N)
        e_p = oracle.l2_error(desc, k, oracle.project_values(desc, k), Q=16, sub=4)
        e_i = oracle.l2_error(desc, k, oracle.interp_values(desc, k), Q=16, sub=4)
        assert e_p <= e_i
        # and no worse than random perturbations of itself
        rng = np.random.default_rng(N)
        c = oracle.project_values(desc, k)
        for _ in range(3):
            c2 = c + rng.normal(scale=1e-3 * np.abs(c).max(), size=c.size)
            assert oracle.l2_error(desc, k, c2, Q=16, sub=4) > e_p


@pytest.mark.parametrize("desc", [GAUSS, LOR, J0], ids=lambda d: d["kind"])
def test_projection_quadrature_converged_at_Q8(desc):
    for N in (256, 1024):
        k = oracle.design(desc, N)
        c8 = oracle.project_values(desc, k, Q=8)
        c16 = oracle.project_values(desc, k, Q=16)
        assert np.abs(c8 - c16).max() <= 1e-13 * np.abs(c16).max()
