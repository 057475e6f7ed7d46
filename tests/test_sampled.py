"""Sampled functions (PWL_F_SAMPLED): f given by FP64 samples on a uniform
grid, f by the cubic through the 4 nearest samples, f'' by the linear
interpolant of the second differences.  The oracle's sampled path is pinned
to the analytic one on cubics (exact) and converges to it at O(h^2) on a
Gaussian; the GPU matches the oracle on the same samples."""
import ctypes

import numpy as np
import pytest

import oracle
from pwl_testutil import DESIGN_REL, EVAL_REL, VALUES_REL, fp32_design_bound, round_knots, round_values

torch = pytest.importorskip("torch")

CUBIC = [0.3, -2.0, 0.5, 1.0]  # 0.3 - 2x + 0.5x^2 + x^3


def _grid(a, b, S):
    return a + (b - a) * np.arange(S) / (S - 1)


def test_oracle_sampled_cubic_is_exact():
    a, b, S = -1.0, 2.0, 50
    d = {"kind": "sampled", "a": a, "b": b, "samples": np.polyval(CUBIC[::-1], _grid(a, b, S))}
    dp = {"kind": "poly", "a": a, "b": b, "p": CUBIC}
    x = np.linspace(a, b, 2001)
    assert np.abs(oracle.f(d, x) - oracle.f(dp, x)).max() <= 1e-13
    f2 = oracle.f2(dp, x)
    assert np.abs(oracle.f2(d, x) - f2).max() <= 1e-10 * np.abs(f2).max()
    assert np.abs(oracle.design(d, 40) - oracle.design(dp, 40)).max() <= 1e-12 * (b - a)
    k = oracle.design(dp, 40)
    for form in ("interp", "project"):
        assert np.abs(oracle.values(d, k, form) - oracle.values(dp, k, form)).max() <= 1e-11


def test_oracle_sampled_gaussian_converges_at_second_order():
    a, b, N = -4.0, 4.0, 64
    dg = {"kind": "gaussian", "a": a, "b": b, "p": [1.0, 0.0, 1.0]}
    ref = oracle.design(dg, N)
    errs = []
    for S in (257, 1025, 4097):
        xs = _grid(a, b, S)
        ds = {"kind": "sampled", "a": a, "b": b, "samples": np.exp(-0.5 * xs * xs)}
        errs.append(np.abs(oracle.design(ds, N) - ref).max())
    # h / 4 per step: the knot error drops by ~16 (O(h^2) second differences)
    assert errs[0] / errs[1] > 10 and errs[1] / errs[2] > 10, errs


def test_sampled_descriptor_checks():
    from paper_1510_02975_gb300 import _capi
    lib = _capi.load()
    f = _capi.PwlFunc()
    fake = ctypes.c_void_p(4096)  # only validated, never dereferenced
    assert lib.pwl_func_sampled(0.0, 1.0, fake, 10, ctypes.byref(f)) == 0
    assert f.kind == 5 and f.p[0] == 10.0
    assert lib.pwl_func_sampled(0.0, 1.0, fake, 3, ctypes.byref(f)) != 0
    assert lib.pwl_func_sampled(1.0, 0.0, fake, 10, ctypes.byref(f)) != 0
    assert lib.pwl_func_sampled(0.0, 1.0, None, 10, ctypes.byref(f)) != 0
    assert lib.pwl_func_sampled(0.0, 1.0, ctypes.c_void_p(4097), 10, ctypes.byref(f)) != 0  # misaligned


@pytest.fixture(scope="module")
def pwl():
    import paper_1510_02975_gb300 as m
    from paper_1510_02975_gb300 import _build
    _build.build()
    return m


def _sampled(a, b, S, fn):
    s = fn(_grid(a, b, S))
    return ({"kind": "sampled", "a": a, "b": b, "samples": torch.tensor(s, dtype=torch.float64, device="cuda")},
            {"kind": "sampled", "a": a, "b": b, "samples": s})


@pytest.mark.gpu
@pytest.mark.parametrize("N", [1, 63, 1024])
def test_sampled_design_values_eval_match_oracle(pwl, N):
    a, b = -10.0, 10.0
    gdesc, odesc = _sampled(a, b, 20001, lambda x: 1.0 / (1.0 + x * x) + 0.1 * np.sin(3 * x))
    knots = pwl.pwl_design(gdesc, N)
    ref = oracle.design(odesc, N)
    kn = knots.cpu().numpy()
    assert np.abs(kn - ref).max() <= DESIGN_REL * (b - a)
    for form in ("interp", "project"):
        vals = pwl.pwl_project(gdesc, knots, form)
        vref = oracle.values(odesc, kn, form)
        assert np.abs(vals.cpu().numpy() - vref).max() <= VALUES_REL * np.abs(vref).max()
        t = pwl.Table(knots, vals)
        x = torch.rand(1 << 18, dtype=torch.float32, device="cuda") * (b - a) + a
        y = t(x).cpu().numpy().astype(np.float64)
        r = oracle.evaluate(round_knots(kn), round_values(vals.cpu().numpy(), "fp32"),
                            x.cpu().numpy().astype(np.float64))
        assert np.abs(y - r).max() <= EVAL_REL * np.abs(r).max()
        t.close()
    # FP32 density mode
    k32 = pwl.pwl_design(gdesc, max(N, 2), 0, "fp32").cpu().numpy()
    ref2 = oracle.design(odesc, max(N, 2))
    assert np.all(np.abs(k32 - ref2) <= fp32_design_bound(ref2))


@pytest.mark.gpu
def test_sampled_in_a_batch_and_error_constants(pwl):
    a, b = 0.0, 50.0
    gdesc, odesc = _sampled(a, b, 50001, lambda x: np.cos(0.3 * x) * np.exp(-0.02 * x))
    cubic_g, cubic_o = _sampled(-1.0, 2.0, 40, lambda x: np.polyval(CUBIC[::-1], x))
    funcs = [{"kind": "gaussian", "a": -4.0, "b": 4.0, "p": [1.0, 0.0, 1.0]}, gdesc, cubic_g]
    ofuncs = [funcs[0], odesc, cubic_o]
    n_int = [300, 777, 50]
    bt = pwl.Batch(funcs, n_int, m_per_interval=16)
    bt.design("fp64")
    bt.project("project")
    kn, vv, off = bt.knots().cpu().numpy(), bt.values().cpu().numpy(), bt.offsets()
    for i, f in enumerate(ofuncs):
        ref = oracle.design(f, n_int[i], 16 * n_int[i])
        assert np.abs(kn[off[i]:off[i + 1]] - ref).max() <= DESIGN_REL * (f["b"] - f["a"]), i
        vref = oracle.values(f, kn[off[i]:off[i + 1]], "project")
        assert np.abs(vv[off[i]:off[i + 1]] - vref).max() <= VALUES_REL * np.abs(vref).max(), i
    bt.close()
    # the integrals of the sampled cubic: f'' = 1 + 6x exactly
    out = pwl.pwl_error_constants(cubic_g, 3000).cpu().numpy()
    ref25 = oracle.integral_abs_f2_pow({"kind": "poly", "a": -1.0, "b": 2.0, "p": CUBIC}, 0.4)
    assert abs(out[1] - ((1 + 6 * 2.0) ** 3 - (1 - 6.0) ** 3) / 18.0) <= 1e-6 * out[1]
    assert abs(out[0] - ref25) <= 1e-5 * ref25  # midpoint rule across the zero of f''
