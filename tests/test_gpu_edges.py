"""Edge cases through the C ABI: empty inputs (no-ops that leave the
gradient outputs untouched), the largest table pwl_table_build accepts
(2^20 - 1 intervals: cells hold ~36 knots each, walked from global memory),
and the size limits of the kernels whose shared-memory state grows with N
(a clean PWL_ENOTSUP, never a launch)."""
import numpy as np
import pytest

import oracle
from pwl_testutil import DESIGN_REL, EVAL_REL, GRAD_REL, round_knots, round_values

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pwl():
    import paper_1510_02975_gb300 as m
    from paper_1510_02975_gb300 import _build
    _build.build()
    return m


@pytest.fixture(scope="module")
def workloads():
    from paper_1510_02975_gb300 import workloads as w
    return w


def test_empty_inputs_are_no_ops(pwl, workloads):
    f = workloads.GAUSSIAN
    kn = pwl.pwl_design(f, 63)
    t = pwl.Table(kn, pwl.pwl_project(f, kn, "project"))
    x0 = torch.empty(0, dtype=torch.float32, device="cuda")
    assert t(x0).numel() == 0
    gv = torch.zeros(64, device="cuda")
    gk = torch.zeros(64, device="cuda")
    assert t.backward(x0, x0, None, gv, gk).numel() == 0
    assert not gv.any() and not gk.any()
    t.close()
    C, N = 8, 16
    knots = torch.linspace(-1, 1, N + 1, device="cuda").repeat(C, 1)
    values = torch.zeros(C, N + 1, device="cuda")
    xr = torch.empty(0, C, device="cuda")
    assert pwl.pwl_channels_forward(knots, values, xr).shape == (0, C)
    gv = torch.zeros_like(values)
    gk = torch.zeros_like(knots)
    assert pwl.pwl_channels_backward(knots, values, xr, xr, None, gv, gk).shape == (0, C)
    assert not gv.any() and not gk.any()


def test_largest_table(pwl, workloads):
    f = workloads.GAUSSIAN
    N = (1 << 20) - 1
    kn = pwl.pwl_design(f, N, 4 * N)
    ref = oracle.design(f, N, 4 * N)
    knots = kn.cpu().numpy()
    assert np.abs(knots - ref).max() <= DESIGN_REL * (f["b"] - f["a"])
    v = pwl.pwl_project(f, kn, "interp")
    t = pwl.Table(kn, v)
    x = workloads.uniform_queries(f, (1 << 20) + 5, seed=1)
    y = t(x).cpu().numpy().astype(np.float64)
    r = oracle.evaluate(round_knots(knots), round_values(v.cpu().numpy(), "fp32"), x.cpu().numpy().astype(np.float64))
    assert np.abs(y - r).max() <= EVAL_REL * np.abs(r).max()
    t.close()


def test_backward_size_limit(pwl, workloads):
    from paper_1510_02975_gb300 import PwlError
    f = workloads.GAUSSIAN
    x = workloads.uniform_queries(f, 1 << 20, seed=1)
    gy = workloads.upstream_grad((x.numel(),), seed=5)
    for N, fits in ((16384, True), (65535, False)):
        kn = pwl.pwl_design(f, N)
        t = pwl.Table(kn, pwl.pwl_project(f, kn, "interp"))
        gv = torch.zeros(N + 1, device="cuda")
        gk = torch.zeros(N + 1, device="cuda")
        if fits:
            gx = t.backward(x, gy, None, gv, gk)
            assert abs(float(gv.double().sum() - gy.double().sum())) <= GRAD_REL * float(gy.double().abs().sum())
            assert abs(float(gk.double().sum() + gx.double().sum())) <= GRAD_REL * float(gx.double().abs().sum())
        else:
            with pytest.raises(PwlError) as e:
                t.backward(x, gy, None, gv, gk)
            assert e.value.status == 4 and "too large" in str(e.value) and "no error" not in str(e.value)
        t.close()


def _tables(C, N, seed):
    # uniform knots on [-8, 8] jittered by up to 0.3 h per channel (well
    # separated: the FP32 backward's delta loses ulp(x) / h of accuracy)
    rng = np.random.default_rng(seed)
    h = 16.0 / N
    knots = np.tile(np.linspace(-8.0, 8.0, N + 1), (C, 1))
    knots[:, 1:-1] += rng.uniform(-0.3, 0.3, (C, N - 1)) * h
    values = rng.normal(size=(C, N + 1))
    return knots.astype(np.float32), values.astype(np.float32)


def test_channel_size_limits(pwl):
    from paper_1510_02975_gb300 import PwlError
    g = torch.Generator(device="cuda").manual_seed(3)
    # forward near its limit (few cells per knot: chains), backward at N = 500
    for N, backward in ((1500, False), (500, True)):
        C, R = 20, 700
        knots, values = _tables(C, N, N)
        kt, vt = torch.tensor(knots, device="cuda"), torch.tensor(values, device="cuda")
        x = torch.randn(R, C, generator=g, device="cuda") * 4.0
        y = pwl.pwl_channels_forward(kt, vt, x).cpu().numpy().astype(np.float64)
        xs = x.cpu().numpy().astype(np.float64)
        for c in range(C):
            r = oracle.evaluate(knots[c].astype(np.float64), values[c].astype(np.float64), xs[:, c])
            assert np.abs(y[:, c] - r).max() <= EVAL_REL * np.abs(r).max(), (N, c)
        if backward:
            gy = torch.randn(R, C, generator=g, device="cuda")
            gv = torch.zeros_like(vt)
            gk = torch.zeros_like(kt)
            gxt = pwl.pwl_channels_backward(kt, vt, x, gy, None, gv, gk)
            gx = gxt.cpu().numpy()
            gys = gy.cpu().numpy().astype(np.float64)
            for c in range(C):
                rgx = oracle.evaluate_grad(knots[c].astype(np.float64), values[c].astype(np.float64),
                                           xs[:, c], gys[:, c])[0]
                assert np.abs(gx[:, c] - rgx).max() <= EVAL_REL * max(np.abs(rgx).max(), 1e-30)
            # the table gradients through the identities sum_j g_v = sum gy and
            # sum_j g_k = -sum g_x (per channel); a bin fed by one or two
            # elements is not held to 1e-5 of its own terms here, since at
            # h = 16/500 FP32 delta carries ~ulp(x) / h ~ 2e-5
            assert bool(((gv.double().sum(1) - gy.double().sum(0)).abs()
                         <= GRAD_REL * gy.double().abs().sum(0)).all())
            assert bool(((gk.double().sum(1) + gxt.double().sum(0)).abs()
                         <= GRAD_REL * gxt.double().abs().sum(0) + 1e-30).all())
    knots, values = _tables(8, 4000, 1)
    with pytest.raises(PwlError) as e:
        pwl.pwl_channels_forward(torch.tensor(knots, device="cuda"), torch.tensor(values, device="cuda"),
                                 torch.zeros(10, 8, device="cuda"))
    assert e.value.status == 4
