"""GPU vs oracle parity through the C ABI: design (Eqs. 16-18), vertex
values (Eqs. 3-6), table evaluation (Algorithm 1) and its backward, on sizes
the oracle finishes quickly that still span many tiles and a ragged tail."""
import numpy as np
import pytest

import oracle
from pwl_testutil import (DESIGN_REL, EVAL_REL, GRAD_REL, VALUES_REL, fp32_design_bound, fp32_integrand_envelope,
                          round_knots, round_values)

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


FUNCS = ["gaussian", "lorentzian", "bessel_j0"]


@pytest.mark.parametrize("name", FUNCS)
@pytest.mark.parametrize("N", [1, 2, 63, 256, 1024, 4096])
def test_design_matches_oracle(pwl, workloads, name, N):
    f = workloads.PAPER_FUNCTIONS[name]
    got = pwl.pwl_design(f, N).cpu().numpy()
    ref = oracle.design(f, N)
    assert np.abs(got - ref).max() <= DESIGN_REL * (f["b"] - f["a"])
    assert got[0] == f["a"] and got[-1] == f["b"]
    assert np.all(np.diff(got) > 0)


@pytest.mark.parametrize("M", [1, 7, 2047, 2048, 2049, 5000])
def test_design_cells_ragged(pwl, workloads, M):
    f = workloads.LORENTZIAN
    N = 40
    got = pwl.pwl_design(f, N, M).cpu().numpy()
    ref = oracle.design(f, N, M)
    assert np.abs(got - ref).max() <= DESIGN_REL * (f["b"] - f["a"])


def test_design_linear_function_is_uniform(pwl):
    f = {"kind": "poly", "a": -1.0, "b": 2.0, "p": [3.0, -0.5]}
    got = pwl.pwl_design(f, 12).cpu().numpy()
    assert np.allclose(got, -1.0 + np.arange(13) * 0.25, atol=1e-15)


@pytest.mark.parametrize("N", [1024, 4096])
def test_design_fp32_density_mode(pwl, workloads, N):
    # FP32 integrand: a relative density error eps moves knot i by about
    # eps N (G(x_i) / G_M) h_i (fp32_design_bound)
    for name in FUNCS:
        f = workloads.PAPER_FUNCTIONS[name]
        got = pwl.pwl_design(f, N, 0, "fp32").cpu().numpy()
        ref = oracle.design(f, N)
        assert np.all(np.abs(got - ref) <= fp32_design_bound(ref)), name


@pytest.mark.parametrize("name", FUNCS)
@pytest.mark.parametrize("form", ["interp", "project"])
@pytest.mark.parametrize("N", [1, 3, 63, 1024, 4096])
def test_values_match_oracle(pwl, workloads, name, form, N):
    f = workloads.PAPER_FUNCTIONS[name]
    knots = pwl.pwl_design(f, N)
    kn = knots.cpu().numpy()
    got = pwl.pwl_project(f, knots, form).cpu().numpy()
    ref = oracle.values(f, kn, form)
    assert np.abs(got - ref).max() <= VALUES_REL * np.abs(ref).max()


@pytest.mark.parametrize("name", FUNCS)
@pytest.mark.parametrize("form", ["interp", "project"])
@pytest.mark.parametrize("N", [63, 1024])
def test_values_fp32_integrand_within_its_rounding(pwl, workloads, name, form, N):
    # FP32 integrand mode against the FP64 oracle on the same knots, within
    # the envelope of FP32 evaluation (pwl_testutil.fp32_integrand_envelope)
    f = workloads.PAPER_FUNCTIONS[name]
    knots = pwl.pwl_design(f, N)
    kn = knots.cpu().numpy()
    got = pwl.pwl_project(f, knots, form, 8, "fp32").cpu().numpy()
    ref = oracle.values(f, kn, form)
    env = fp32_integrand_envelope(f)
    err = np.abs(got - ref).max()
    assert err <= 2.5 * env, (err, env)
    # and not FP64-exact by accident: the mode's rounding is visible
    assert err > 0.0


def test_projection_large_n_global_solver(pwl, workloads):
    # N + 1 > rows that fit in shared memory: the solver runs on global scratch
    f = workloads.BESSEL_J0
    N = 20000
    knots = pwl.pwl_design(f, N)
    kn = knots.cpu().numpy()
    got = pwl.pwl_project(f, knots, "project").cpu().numpy()
    ref = oracle.values(f, kn, "project")
    assert np.abs(got - ref).max() <= VALUES_REL * np.abs(ref).max()


def _table_and_ref(pwl, f, N, form="project", dtype="fp32", k_cells=0):
    knots = pwl.pwl_design(f, N)
    vals = pwl.pwl_project(f, knots, form)
    t = pwl.Table(knots, vals, dtype, k_cells)
    xk = round_knots(knots.cpu().numpy())
    vk = round_values(vals.cpu().numpy(), dtype)
    return t, xk, vk


def _check_eval(y, xk, vk, x):
    ref = oracle.evaluate(xk, vk, x.cpu().numpy().astype(np.float64))
    got = y.cpu().numpy().astype(np.float64)
    nan = np.isnan(ref)
    assert np.array_equal(nan, np.isnan(got))
    assert np.abs(got[~nan] - ref[~nan]).max(initial=0.0) <= EVAL_REL * np.abs(ref[~nan]).max(initial=1.0)


@pytest.mark.parametrize("name", FUNCS)
@pytest.mark.parametrize("N", [1, 63, 256, 1024, 4096])
def test_eval_matches_oracle(pwl, workloads, name, N):
    f = workloads.PAPER_FUNCTIONS[name]
    t, xk, vk = _table_and_ref(pwl, f, N)
    m = (1 << 20) + 3  # several tiles and a ragged tail
    x = workloads.uniform_queries(f, m, seed=1)
    _check_eval(t(x), xk, vk, x)
    xn = workloads.normal_queries(f, m, seed=2)
    _check_eval(t(xn), xk, vk, xn)
    t.close()


def test_eval_small_case_both_forms(pwl, workloads):
    s = workloads.SMALL
    for form in ("interp", "project"):
        t, xk, vk = _table_and_ref(pwl, s["func"], s["n_intervals"], form)
        x = workloads.uniform_queries(s["func"], s["m"], s["seed"])
        _check_eval(t(x), xk, vk, x)
        t.close()


@pytest.mark.parametrize("k_cells", [1, 3, 17, 64, 1000, 9000])
def test_eval_any_cell_count(pwl, workloads, k_cells):
    # few cells force chains of many knots per cell; many cells none; both
    # cell indexes (modes 2 and 3) are checked whichever pwl_eval picks
    f = workloads.LORENTZIAN
    t, xk, vk = _table_and_ref(pwl, f, 300, k_cells=k_cells)
    assert t.info["k_cells"] == k_cells
    x = workloads.uniform_queries(f, 100003, seed=7)
    x[:xk.size] = torch.tensor(xk, dtype=torch.float32, device="cuda")
    _check_eval(t(x), xk, vk, x)
    for mode in (2, 3, 6):
        y = t.variant(mode, x)
        _check_eval(y, xk, vk, x)
        # exact at the knots in every index
        assert np.array_equal(y[:xk.size].cpu().numpy().astype(np.float64), vk)
    t.close()


@pytest.mark.parametrize("name", FUNCS)
@pytest.mark.parametrize("N", [64, 1024, 4096])
def test_eval_both_layouts_default_cells(pwl, workloads, name, N):
    f = workloads.PAPER_FUNCTIONS[name]
    t, xk, vk = _table_and_ref(pwl, f, N)
    x = workloads.normal_queries(f, (1 << 19) + 9, seed=4)
    for mode in (2, 3, 6):
        _check_eval(t.variant(mode, x), xk, vk, x)
    t.close()


def test_compact_side_records_for_the_largest_chain_free_index(pwl, workloads):
    # the Lorentzian at N = 4096 needs ~20 K cells for a chain-free index:
    # with one side record per knot it fits the one-CTA budget (layout 2);
    # every lookup side of every knot matches the oracle, and layout 2 gives
    # the same bits as the two-side-record index (mode 2) on the same cells
    f = workloads.LORENTZIAN
    t, xk, vk = _table_and_ref(pwl, f, 4096)
    assert int(t.info["layout"]) == 2 and int(t.info["n_chain"]) == 0
    assert t.info["eval_smem_bytes"] <= 190 * 1024
    x = workloads.uniform_queries(f, (1 << 20) + 5, seed=3)
    x[:xk.size] = torch.tensor(xk, dtype=torch.float32, device="cuda")
    mids = 0.5 * (xk[1:] + xk[:-1])
    x[xk.size:xk.size + mids.size] = torch.tensor(mids, dtype=torch.float32, device="cuda")
    nb = np.nextafter(xk.astype(np.float32), np.float32(-np.inf))
    x[xk.size + mids.size:2 * xk.size + mids.size] = torch.tensor(nb, device="cuda")
    y = t(x)
    _check_eval(y, xk, vk, x)
    assert np.array_equal(y[:xk.size].cpu().numpy().astype(np.float64), vk)
    assert torch.equal(y, t.variant(2, x))
    assert torch.equal(y, t.variant(6, x))
    t.close()


def test_eval_edge_cases(pwl, workloads):
    f = workloads.BESSEL_J0
    t, xk, vk = _table_and_ref(pwl, f, 257)
    x = np.concatenate([xk, [-1e30, -1.0, 0.0, 50.0, 51.0, 1e30, np.nan, np.inf, -np.inf],
                        0.5 * (xk[1:] + xk[:-1]), np.nextafter(xk.astype(np.float32), np.float32(np.inf))])
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    _check_eval(t(xt), xk, vk, xt)
    # exact at the knots
    yk = t(torch.tensor(xk, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert np.array_equal(yk.astype(np.float64), vk)
    # m = 0, 1, 3 and unaligned pointers
    for m in (0, 1, 3, 5):
        xs = torch.linspace(-1, 51, m, device="cuda")
        _check_eval(t(xs), xk, vk, xs)
    big = workloads.uniform_queries(f, 4099, seed=3)
    for off_x, off_y in ((1, 1), (1, 2), (3, 0), (0, 2)):
        xs = big[off_x:off_x + 4000]
        out = torch.empty(4100, device="cuda")
        ys = out[off_y:off_y + 4000]
        pwl.pwl_eval(t.handle, xs, ys)
        _check_eval(ys, xk, vk, xs)
    # in place
    xs = big.clone()
    pwl.pwl_eval(t.handle, xs, xs)
    _check_eval(xs, xk, vk, big)
    t.close()


@pytest.mark.parametrize("dtype", ["bf16", "fp16"])
def test_reduced_precision_tables(pwl, workloads, dtype):
    for name in FUNCS:
        f = workloads.PAPER_FUNCTIONS[name]
        t, xk, vk = _table_and_ref(pwl, f, 1024, dtype=dtype)
        x = workloads.uniform_queries(f, 1 << 18, seed=1)
        _check_eval(t(x), xk, vk, x)
        t.close()


@pytest.mark.parametrize("io", ["bf16", "fp16"])
def test_reduced_precision_io(pwl, workloads, io):
    tdt = {"bf16": torch.bfloat16, "fp16": torch.float16}[io]
    f = workloads.GAUSSIAN
    t, xk, vk = _table_and_ref(pwl, f, 1024)
    x = workloads.uniform_queries(f, (1 << 18) + 5, seed=1).to(tdt)
    y = t(x)
    ref = oracle.evaluate(xk, vk, x.float().cpu().numpy().astype(np.float64))
    got = y.float().cpu().numpy().astype(np.float64)
    # output rounded once to the 16-bit type: half an ulp of |y| plus the FP32 bound
    # (relative ulp <= 2^-7 for bf16, 2^-10 for fp16; 2^-24 covers fp16 subnormals)
    ulp = {"bf16": 2.0**-7, "fp16": 2.0**-10}[io]
    assert np.all(np.abs(got - ref) <= 0.5 * ulp * np.abs(ref) * 1.0001 + EVAL_REL * np.abs(ref).max() + 2.0**-24)
    t.close()


def test_variant_binary_search(pwl, workloads):
    for name in FUNCS:
        f = workloads.PAPER_FUNCTIONS[name]
        t, xk, vk = _table_and_ref(pwl, f, 1024)
        x = workloads.uniform_queries(f, (1 << 18) + 1, seed=1)
        _check_eval(t.variant(0, x), xk, vk, x)
        t.close()


def test_variant_texture_filter(pwl, workloads):
    # the filter weight has 8 fractional bits: |err| <= |v_i - v_{i-1}| / 2^8
    # (plus FP32 rounding of the coordinate and the result)
    for name in FUNCS:
        f = workloads.PAPER_FUNCTIONS[name]
        t, xk, vk = _table_and_ref(pwl, f, 1024)
        x = workloads.uniform_queries(f, (1 << 18) + 1, seed=1)
        y = t.variant(1, x).cpu().numpy().astype(np.float64)
        xs = x.cpu().numpy().astype(np.float64)
        ref = oracle.evaluate(xk, vk, xs)
        i = np.clip(np.searchsorted(xk, xs, side="right"), 1, len(xk) - 1)
        dv = np.abs(vk[i] - vk[i - 1])
        assert np.all(np.abs(y - ref) <= dv / 256.0 + 1e-6 * np.abs(vk).max())
        t.close()


@pytest.mark.parametrize("name", FUNCS)
@pytest.mark.parametrize("N", [1, 5, 256, 4096])
def test_backward_matches_oracle(pwl, workloads, name, N):
    f = workloads.PAPER_FUNCTIONS[name]
    t, xk, vk = _table_and_ref(pwl, f, N)
    m = (1 << 18) + 7
    x = workloads.uniform_queries(f, m, seed=1)
    # some queries outside the domain and exactly at knots
    x[:100] = float(f["a"]) - 1.0
    x[100:200] = float(f["b"]) + 1.0
    x[200:200 + len(xk)] = torch.tensor(xk, dtype=torch.float32, device="cuda")
    gy = workloads.upstream_grad((m,), seed=5)
    gv = torch.zeros(N + 1, device="cuda")
    gk = torch.zeros(N + 1, device="cuda")
    gx = t.backward(x, gy, None, gv, gk)
    rgx, rgv, rgk, rgva, rgka = oracle.evaluate_grad(xk, vk, x.cpu().numpy().astype(np.float64),
                                                     gy.cpu().numpy().astype(np.float64))
    assert np.abs(gx.cpu().numpy() - rgx).max() <= EVAL_REL * np.abs(rgx).max()
    assert np.all(np.abs(gv.cpu().numpy() - rgv) <= GRAD_REL * rgva + 1e-30)
    assert np.all(np.abs(gk.cpu().numpy() - rgk) <= GRAD_REL * rgka + 1e-30)
    # a second call agrees to FP32 rounding of the in-CTA sums
    gv2 = torch.zeros_like(gv)
    gk2 = torch.zeros_like(gk)
    gx2 = t.backward(x, gy, None, gv2, gk2)
    assert torch.equal(gx, gx2)
    assert np.all(np.abs((gv2 - gv).cpu().numpy()) <= GRAD_REL * rgva + 1e-30)
    assert np.all(np.abs((gk2 - gk).cpu().numpy()) <= GRAD_REL * rgka + 1e-30)
    t.close()


def _backward_vs_oracle(t, xk, vk, x, gy, N):
    gv = torch.zeros(N + 1, device="cuda")
    gk = torch.zeros(N + 1, device="cuda")
    gx = t.backward(x, gy, None, gv, gk)
    rgx, rgv, rgk, rgva, rgka = oracle.evaluate_grad(xk, vk, x.cpu().numpy().astype(np.float64),
                                                     gy.cpu().numpy().astype(np.float64))
    return gx.cpu().numpy(), gv.cpu().numpy(), gk.cpu().numpy(), (rgx, rgv, rgk, rgva, rgka)


@pytest.mark.parametrize("N", [1, 5, 4096])
def test_backward_fixed_point_wraps_and_wide_terms(pwl, workloads, N):
    # The in-CTA sums are int32 fixed point whose unit each CTA takes from
    # the |gy| of its first vectors.  Tiny gradients there and O(1) ones
    # after them put later terms at up to ~2^31 units: most adds wrap (their
    # +-2^32 units go to the CTA row) and the largest terms leave the int32
    # range (FP32 path); runs of one sign drive the wraps both ways.
    f = workloads.GAUSSIAN
    t, xk, vk = _table_and_ref(pwl, f, N)
    m = (1 << 22) + 5
    x = workloads.uniform_queries(f, m, seed=3)
    g = torch.Generator(device="cuda").manual_seed(8)
    sign = torch.where(torch.arange(m, device="cuda") // 50000 % 2 == 0, 1.0, -1.0)
    gy = sign * (0.5 + torch.rand(m, generator=g, device="cuda"))
    gy[: 1 << 20] *= 2.0 ** -9
    gx, gv, gk, (rgx, rgv, rgk, rgva, rgka) = _backward_vs_oracle(t, xk, vk, x, gy, N)
    assert np.abs(gx - rgx).max() <= EVAL_REL * np.abs(rgx).max()
    assert np.all(np.abs(gv - rgv) <= GRAD_REL * rgva + 1e-30)
    assert np.all(np.abs(gk - rgk) <= GRAD_REL * rgka + 1e-30)
    t.close()


@pytest.mark.parametrize("N", [5, 1024])
def test_backward_gradients_spanning_many_decades(pwl, workloads, N):
    # |gy| log-uniform over 1e-15 .. 1e15: the fixed-point unit follows the
    # geometric mean, the large terms take the FP32 path, the tiny ones round
    # to a unit that is far below the knots' sums of |terms|
    f = workloads.LORENTZIAN
    t, xk, vk = _table_and_ref(pwl, f, N)
    m = (1 << 20) + 3
    x = workloads.uniform_queries(f, m, seed=4)
    g = torch.Generator(device="cuda").manual_seed(9)
    mag = 10.0 ** (30.0 * torch.rand(m, generator=g, device="cuda") - 15.0)
    gy = (workloads.upstream_grad((m,), seed=6).sign() * mag).float()
    gx, gv, gk, (rgx, rgv, rgk, rgva, rgka) = _backward_vs_oracle(t, xk, vk, x, gy, N)
    assert np.all(np.abs(gx - rgx) <= 2.0 ** -23 * np.abs(rgx) + 1e-37)
    assert np.all(np.abs(gv - rgv) <= GRAD_REL * rgva + 1e-30)
    assert np.all(np.abs(gk - rgk) <= GRAD_REL * rgka + 1e-30)
    t.close()


def test_backward_unit_from_an_empty_sample(pwl, workloads):
    # zero gradients in every thread's first vector (no exponent sample: the
    # default unit 2^-23) and N(0, 1) ones after them
    f = workloads.BESSEL_J0
    N = 1024
    t, xk, vk = _table_and_ref(pwl, f, N)
    m = (1 << 22) + 9
    x = workloads.uniform_queries(f, m, seed=14)
    gy = workloads.upstream_grad((m,), seed=15)
    gy[: 1 << 20] = 0.0
    gx, gv, gk, (rgx, rgv, rgk, rgva, rgka) = _backward_vs_oracle(t, xk, vk, x, gy, N)
    assert np.abs(gx - rgx).max() <= EVAL_REL * np.abs(rgx).max()
    assert np.all(np.abs(gv - rgv) <= GRAD_REL * rgva + 1e-30)
    assert np.all(np.abs(gk - rgk) <= GRAD_REL * rgka + 1e-30)
    t.close()


@pytest.mark.parametrize("scale", [1e-28, 1e28])
def test_backward_gradients_of_extreme_magnitude(pwl, workloads, scale):
    # gy ~ N(0, 1) * 1e-28: the fixed-point unit 2^-117, still 2^-23 of the
    # typical term; * 1e28: every term is 2^31 units or more and takes the
    # exact 64-bit split (low 32 bits in shared memory, multiples of 2^32
    # units in the row)
    f = workloads.GAUSSIAN
    N = 1024
    t, xk, vk = _table_and_ref(pwl, f, N)
    m = (1 << 21) + 3
    x = workloads.uniform_queries(f, m, seed=16)
    gy = workloads.upstream_grad((m,), seed=17) * scale
    gx, gv, gk, (rgx, rgv, rgk, rgva, rgka) = _backward_vs_oracle(t, xk, vk, x, gy, N)
    assert np.abs(gx - rgx).max() <= EVAL_REL * np.abs(rgx).max()
    assert np.all(np.abs(gv - rgv) <= GRAD_REL * rgva)
    assert np.all(np.abs(gk - rgk) <= GRAD_REL * rgka)
    t.close()


def test_backward_zero_and_non_finite_gradients(pwl, workloads):
    f = workloads.GAUSSIAN
    N = 256
    t, xk, vk = _table_and_ref(pwl, f, N)
    m = (1 << 18) + 1
    x = workloads.uniform_queries(f, m, seed=2)
    # all-zero upstream gradient: every output exactly zero
    gx, gv, gk, _ = _backward_vs_oracle(t, xk, vk, x, torch.zeros(m, device="cuda"), N)
    assert not gx.any() and not gv.any() and not gk.any()
    # one inf and one NaN among normal gradients, at queries strictly inside
    # intervals: the knots of those intervals become non-finite like the
    # FP64 reference, every other knot keeps its value
    gy = workloads.upstream_grad((m,), seed=5)
    xs = x.cpu().numpy().astype(np.float64)
    i = np.clip(np.searchsorted(xk, xs, side="right"), 1, N)
    inside = np.flatnonzero((xs > xk[i - 1]) & (xs < xk[i]))
    q_inf, q_nan = int(inside[1000]), int(inside[-1000])
    gy[q_inf] = float("inf")
    gy[q_nan] = float("nan")
    gx, gv, gk, (rgx, rgv, rgk, rgva, rgka) = _backward_vs_oracle(t, xk, vk, x, gy, N)
    for got, ref, refa in ((gv, rgv, rgva), (gk, rgk, rgka)):
        fin = np.isfinite(ref)
        assert not fin.all()
        assert np.array_equal(np.isfinite(got), fin)
        assert np.array_equal(np.isnan(got), np.isnan(ref))
        assert np.all(np.abs(got[fin] - ref[fin]) <= GRAD_REL * refa[fin] + 1e-30)
    assert np.isinf(gx[q_inf]) and np.isnan(gx[q_nan])
    t.close()


@pytest.mark.parametrize("N", [256, 4096])
def test_backward_table_gradients_reproducible(pwl, workloads, N):
    # Interior queries and gradients of moderate range: the in-CTA sums are
    # integers (order-independent), the only FP32 terms of a CTA's row are
    # wraps (exact multiples of the unit's 2^32), each CTA's unit comes from
    # the same gy values on every call, and the rows are reduced in a fixed
    # order, so two calls give the same table gradients bit for bit.
    f = workloads.LORENTZIAN
    t, xk, vk = _table_and_ref(pwl, f, N)
    m = (1 << 22) + 1
    x = workloads.uniform_queries(f, m, seed=12)
    x[x == float(f["a"])] = 0.0  # strictly inside (a, b): no end sums
    gy = workloads.upstream_grad((m,), seed=13)
    out = []
    for _ in range(2):
        gv, gk = torch.zeros(N + 1, device="cuda"), torch.zeros(N + 1, device="cuda")
        gx = t.backward(x, gy, None, gv, gk)
        out.append((gx, gv, gk))
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2], out[1][2])
    _, rgv, rgk, rgva, rgka = oracle.evaluate_grad(xk, vk, x.cpu().numpy().astype(np.float64),
                                                   gy.cpu().numpy().astype(np.float64))
    assert np.all(np.abs(out[0][1].cpu().numpy() - rgv) <= GRAD_REL * rgva + 1e-30)
    assert np.all(np.abs(out[0][2].cpu().numpy() - rgk) <= GRAD_REL * rgka + 1e-30)
    t.close()


def test_backward_in_place_and_unaligned(pwl, workloads):
    # gx may alias gy: the in-place call gives the out-of-place gx bit for bit
    # (each CTA's fixed-point unit comes from gy values that only the thread
    # which overwrites them reads first) and the same table gradients; odd
    # offsets take the scalar path
    f = workloads.BESSEL_J0
    N = 1024
    t, xk, vk = _table_and_ref(pwl, f, N)
    m = (1 << 20) + 3
    x = workloads.uniform_queries(f, m, seed=7)
    gy = workloads.upstream_grad((m,), seed=8)
    gv, gk = torch.zeros(N + 1, device="cuda"), torch.zeros(N + 1, device="cuda")
    gx = t.backward(x, gy, None, gv, gk)
    g2 = gy.clone()
    gv2, gk2 = torch.zeros_like(gv), torch.zeros_like(gk)
    t.backward(x, g2, g2, gv2, gk2)
    assert torch.equal(g2, gx)
    _, _, _, rgva, rgka = oracle.evaluate_grad(xk, vk, x.cpu().numpy().astype(np.float64),
                                               gy.cpu().numpy().astype(np.float64))
    assert np.all(np.abs((gv2 - gv).cpu().numpy()) <= GRAD_REL * rgva + 1e-30)
    assert np.all(np.abs((gk2 - gk).cpu().numpy()) <= GRAD_REL * rgka + 1e-30)
    for off in (1, 3):
        xs, gs = x[off:off + 400001], gy[off:off + 400001]
        gvo, gko = torch.zeros_like(gv), torch.zeros_like(gk)
        gxo = t.backward(xs, gs, None, gvo, gko)
        rgx, rgv, rgk, rgva, rgka = oracle.evaluate_grad(xk, vk, xs.cpu().numpy().astype(np.float64),
                                                         gs.cpu().numpy().astype(np.float64))
        assert np.abs(gxo.cpu().numpy() - rgx).max() <= EVAL_REL * np.abs(rgx).max()
        assert np.all(np.abs(gvo.cpu().numpy() - rgv) <= GRAD_REL * rgva + 1e-30)
        assert np.all(np.abs(gko.cpu().numpy() - rgk) <= GRAD_REL * rgka + 1e-30)
    t.close()


def _sorted_and_clustered_sets(xk, m, g):
    """Query sets whose warps fall in one or two intervals (the warp-aggregated
    scatter) next to warps that do not: sorted uniform queries, one interval,
    two adjacent intervals in sorted blocks, sorted queries with clamped and
    out-of-domain ones sprinkled in, and random queries with a point mass
    inside an interval or at a knot."""
    a, b = float(xk[0]), float(xk[-1])
    k = len(xk) // 2
    x0, x1, x2 = float(xk[k - 1]), float(xk[k]), float(xk[k + 1])
    u = torch.rand(m, generator=g, dtype=torch.float64, device="cuda")
    sets = {
        "sorted": torch.sort((a + (b - a) * u).float()).values,
        "one_interval": (x1 + (x2 - x1) * 0.999 * u).float(),
        "two_intervals": torch.sort((x0 + (x2 - x0) * 0.999 * u).float()).values,
    }
    mixed = sets["sorted"].clone()
    idx = torch.randint(0, m, (m // 500,), generator=g, device="cuda")
    mixed[idx] = torch.tensor([a - 1.0, b + 1.0, a, b], device="cuda").repeat(len(idx) // 4 + 1)[:len(idx)]
    sets["sorted_with_ends"] = mixed
    # point masses scattered through a random stream (the hot-interval sums):
    # half the queries inside one interval, and 30% exactly at a knot
    u32 = (a + (b - a) * u).float()
    pm = u32.clone()
    pm[torch.rand(m, generator=g, device="cuda") < 0.5] = float(0.5 * (x1 + x2))
    sets["point_mass"] = pm
    pk = u32.clone()
    pk[torch.rand(m, generator=g, device="cuda") < 0.3] = x1
    sets["point_mass_at_knot"] = pk
    return sets


@pytest.mark.parametrize("N", [256, 4096])
def test_backward_sorted_and_clustered_queries(pwl, workloads, N):
    f = workloads.GAUSSIAN
    t, xk, vk = _table_and_ref(pwl, f, N)
    # ~7 vectors per thread: warps switch between the per-lane and the
    # aggregated scatter several times
    m = (1 << 22) + 13
    g = torch.Generator(device="cuda").manual_seed(21)
    gy = workloads.upstream_grad((m,), seed=5)
    gys = gy.cpu().numpy().astype(np.float64)
    for name, x in _sorted_and_clustered_sets(xk, m, g).items():
        gv = torch.zeros(N + 1, device="cuda")
        gk = torch.zeros(N + 1, device="cuda")
        gx = t.backward(x, gy, None, gv, gk)
        rgx, rgv, rgk, rgva, rgka = oracle.evaluate_grad(xk, vk, x.cpu().numpy().astype(np.float64), gys)
        assert np.abs(gx.cpu().numpy() - rgx).max() <= EVAL_REL * np.abs(rgx).max(), name
        assert np.all(np.abs(gv.cpu().numpy() - rgv) <= GRAD_REL * rgva + 1e-30), name
        assert np.all(np.abs(gk.cpu().numpy() - rgk) <= GRAD_REL * rgka + 1e-30), name
    t.close()


@pytest.mark.parametrize("name", FUNCS)
@pytest.mark.parametrize("N", [7, 260, 2596])
def test_uniform_partition_table(pwl, workloads, name, N):
    # the uniform partition's lookup: two cells per interval put at most one
    # knot in a cell whichever way FP32 rounds it, and pwl_eval serves the
    # table from the 16-byte index without chains
    f = workloads.PAPER_FUNCTIONS[name]
    a, b = f["a"], f["b"]
    kn = a + (b - a) * torch.arange(N + 1, dtype=torch.float64, device="cuda") / N
    kn[-1] = b
    vals = pwl.pwl_project(f, kn, "project")
    t = pwl.Table(kn, vals, "fp32", 2 * N)
    assert int(t.info["layout"]) == 1 and int(t.info["n_chain"]) == 0
    x = workloads.uniform_queries(f, (1 << 20) + 3, seed=1)
    x[: N + 1] = torch.tensor(round_knots(kn.cpu().numpy()), dtype=torch.float32, device="cuda")
    _check_eval(t(x), round_knots(kn.cpu().numpy()), round_values(vals.cpu().numpy(), "fp32"), x)
    t.close()


def test_invalid_arguments_are_rejected(pwl, workloads):
    from paper_1510_02975_gb300 import PwlError
    bad = dict(workloads.GAUSSIAN, a=1.0, b=0.0)
    with pytest.raises(PwlError):
        pwl.pwl_design(bad, 10)
    k = torch.tensor([0.0, 1.0, 1.0, 2.0], dtype=torch.float64, device="cuda")
    with pytest.raises(PwlError):
        pwl.Table(k, torch.zeros_like(k))
    k = torch.tensor([0.0, 1.0, 2.0], dtype=torch.float64, device="cuda")
    v = torch.tensor([0.0, float("nan"), 2.0], dtype=torch.float64, device="cuda")
    with pytest.raises(PwlError):
        pwl.Table(k, v)


def test_table_update_in_place(pwl, workloads):
    # rebuild a table from new knots and values (same N): results follow the new function
    f1, f2 = workloads.GAUSSIAN, dict(workloads.GAUSSIAN, p=[2.0, 0.5, 0.7])
    N = 512
    k1 = pwl.pwl_design(f1, N)
    t = pwl.Table(k1, pwl.pwl_project(f1, k1, "project"))
    x = workloads.uniform_queries(f2, 300001, seed=9)
    t.variant(1, x)  # creates the texture of the comparison path from the first function
    k2 = pwl.pwl_design(f2, N)
    v2 = pwl.pwl_project(f2, k2, "project")
    # on a non-blocking stream: the texture refresh must follow the update there
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        t.update(k2, v2)
        y_tex = t.variant(1, x)
    torch.cuda.current_stream().wait_stream(s)
    pwl.pwl_table_check(t.handle)
    xk, vk = round_knots(k2.cpu().numpy()), round_values(v2.cpu().numpy(), "fp32")
    _check_eval(t(x), xk, vk, x)
    for mode in (2, 3, 6):
        _check_eval(t.variant(mode, x), xk, vk, x)
    # the texture filter follows the new values (8-bit weight bound)
    xs = x.cpu().numpy().astype(np.float64)
    ref = oracle.evaluate(xk, vk, xs)
    i = np.clip(np.searchsorted(xk, xs, side="right"), 1, len(xk) - 1)
    dv = np.abs(vk[i] - vk[i - 1])
    y = y_tex.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(y - ref) <= dv / 256.0 + 1e-6 * np.abs(vk).max())
    t.close()


def test_table_update_moving_an_end_knot_is_reported(pwl, workloads):
    # the cell grids of a table span the built [x_0, x_N]: an update that
    # moves an end knot is flagged by pwl_table_check, and a valid update
    # afterwards clears the flag
    f = workloads.GAUSSIAN
    N = 256
    k = pwl.pwl_design(f, N)
    v = pwl.pwl_project(f, k, "project")
    t = pwl.Table(k, v)
    for end in (0, N):
        k2 = k.clone()
        k2[end] += 0.25 * float(k[1] - k[0]) * (1 if end == 0 else -1)
        t.update(k2, v)
        with pytest.raises(pwl.PwlError, match="end knots"):
            pwl.pwl_table_check(t.handle)
    t.update(k, v)
    pwl.pwl_table_check(t.handle)
    x = workloads.uniform_queries(f, 100003, seed=2)
    _check_eval(t(x), round_knots(k.cpu().numpy()), round_values(v.cpu().numpy(), "fp32"), x)
    t.close()


def test_design_projection_update_eval_in_a_cuda_graph(pwl, workloads):
    # the asynchronous calls (design, projection, table update, evaluation)
    # allocate nothing and never synchronize, so a stream capture replays them
    f = workloads.BESSEL_J0
    N = 1024
    knots = pwl.pwl_design(f, N)
    vals = pwl.pwl_project(f, knots, "project")
    t = pwl.Table(knots, vals)
    lib = __import__("paper_1510_02975_gb300._capi", fromlist=["load"]).load()
    wsd = torch.empty(lib.pwl_design_workspace_size(N, 0), dtype=torch.uint8, device="cuda")
    wsp = torch.empty(lib.pwl_project_workspace_size(N), dtype=torch.uint8, device="cuda")
    x = workloads.uniform_queries(f, 1 << 20, seed=3)
    y = torch.empty_like(x)

    def body():
        pwl.pwl_design(f, N, 0, "fp64", knots=knots, workspace=wsd)
        pwl.pwl_project(f, knots, "project", values=vals, workspace=wsp)
        t.update(knots, vals)
        pwl.pwl_eval(t.handle, x, y)

    body()
    torch.cuda.synchronize()
    y_eager = y.clone()
    k_eager = knots.clone()
    knots.zero_()
    vals.zero_()
    y.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            body()
    torch.cuda.current_stream().wait_stream(s)
    knots.zero_()
    y.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(knots, k_eager)
    assert torch.equal(y, y_eager)
    t.close()


@pytest.mark.parametrize("N,k_cells", [(256, 0), (4096, 0), (300, 40)])
def test_eval_synthetic_checksum_matches_oracle(pwl, workloads, N, k_cells):
    # compute-ceiling mode: the generated queries are rebuilt on the host from
    # the same hash; the GPU checksum of Algorithm 1 over them equals the
    # oracle's sum within the FP32 evaluation bound plus FP32 summation
    # (every thread sums its share in FP32)
    f = workloads.PAPER_FUNCTIONS["lorentzian"]
    t, xk, vk = _table_and_ref(pwl, f, N, "project", "fp32", k_cells)
    m, seed = (1 << 20) + 7, 12345
    got = pwl.pwl_eval_synthetic(t.handle, m, seed).item()
    x = workloads.synthetic_queries(float(t.info["a"]), float(t.info["b"]), m, seed).astype(np.float64)
    ref_y = oracle.evaluate(xk, vk, x)
    ref = float(np.sum(ref_y))
    bound = m * EVAL_REL * np.abs(vk).max() + 1e-5 * float(np.sum(np.abs(ref_y)))
    assert abs(got - ref) <= bound
    t.close()
