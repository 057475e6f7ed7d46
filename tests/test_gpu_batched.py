"""GPU vs oracle parity of the batched path: many independent functions with
uneven knot and query counts designed (Eqs. 16-18), projected (Eqs. 3-6),
indexed and evaluated (Algorithm 1) through the pwl_batch_* calls."""
import numpy as np
import pytest

import oracle
from pwl_testutil import DESIGN_REL, EVAL_REL, VALUES_REL, fp32_design_bound, fp32_integrand_envelope, round_knots

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


def _batch_inputs(workloads, F, seed, knots_hi=700, q_hi=2e5):
    """Functions of the batched workload's families at small sizes, N from 1
    up, a few functions without queries, query counts from 1 (ragged) to
    q_hi; queries uniform on each domain widened by 10% on both sides
    (clamping), one NaN."""
    funcs, n_int, n_q = workloads.batch_functions(F, seed=seed, knots_lo=2, knots_hi=knots_hi, q_lo=1, q_hi=q_hi)
    n_int[0] = 1
    n_int[1] = 2
    n_q[2] = 0
    n_q[3] = 1
    n_q[5] = 0
    rng = np.random.default_rng(seed)
    xs = []
    for f, nq in zip(funcs, n_q):
        w = f["b"] - f["a"]
        xs.append(rng.uniform(f["a"] - 0.1 * w, f["b"] + 0.1 * w, nq).astype(np.float32))
    qo = np.concatenate([[0], np.cumsum(n_q)]).astype(np.int64)
    x = np.concatenate(xs)
    if x.size > 10:
        x[7] = np.nan
    return funcs, n_int, qo, x


def _check_batch_eval(b, funcs, qo, x, y):
    xk = b.knots_fp32().cpu().numpy().astype(np.float64)
    vk = b.values_fp32().cpu().numpy().astype(np.float64)
    off = b.offsets()
    for f in range(len(funcs)):
        q0, q1 = int(qo[f]), int(qo[f + 1])
        if q1 == q0:
            continue
        kn, vv = xk[off[f]:off[f + 1]], vk[off[f]:off[f + 1]]
        ref = oracle.evaluate(kn, vv, x[q0:q1].astype(np.float64))
        got = y[q0:q1].astype(np.float64)
        assert np.array_equal(np.isnan(ref), np.isnan(got)), f
        ok = ~np.isnan(ref)
        assert np.abs(got[ok] - ref[ok]).max() <= EVAL_REL * np.abs(vv).max(), f


@pytest.mark.parametrize("form,F", [("interp", 40), ("project", 40), ("project", 70)])
def test_batch_design_values_eval_match_oracle(pwl, workloads, form, F):
    # F = 40: one CTA per function solves the Gram system (cyclic reduction);
    # F = 70: one warp per function (partitioned Thomas)
    funcs, n_int, qo, x = _batch_inputs(workloads, F, seed=11)
    mper = 16
    b = pwl.Batch(funcs, n_int, m_per_interval=mper)
    b.design()
    b.project(form)
    b.build()
    b.check()
    knots = b.knots().cpu().numpy()
    vals = b.values().cpu().numpy()
    off = b.offsets()
    for i, f in enumerate(funcs):
        kn = knots[off[i]:off[i + 1]]
        ref = oracle.design(f, n_int[i], mper * n_int[i])
        assert np.abs(kn - ref).max() <= DESIGN_REL * (f["b"] - f["a"]), i
        vref = oracle.values(f, kn, form)
        assert np.abs(vals[off[i]:off[i + 1]] - vref).max() <= VALUES_REL * np.abs(vref).max(), i
    # the index's FP32 tables are the FP64 ones rounded to nearest
    assert np.array_equal(b.knots_fp32().cpu().numpy().astype(np.float64), round_knots(knots))
    assert np.array_equal(b.values_fp32().cpu().numpy().astype(np.float64), round_knots(vals))
    xd = torch.tensor(x, device="cuda")
    b.plan(qo)
    y = b.eval(xd).cpu().numpy()
    _check_batch_eval(b, funcs, qo, x, y)
    b.close()


@pytest.mark.parametrize("F", [40, 70])
def test_batch_fp32_projection_within_integrand_rounding(pwl, workloads, F):
    # FP32 integrand mode with both solvers (F = 40: cyclic reduction, one
    # CTA per function; F = 70: partitioned Thomas, one warp per function)
    # against the oracle's P_T values on the same knots
    funcs, n_int, _, _ = _batch_inputs(workloads, F, seed=21)
    b = pwl.Batch(funcs, n_int, m_per_interval=16)
    b.design()
    b.project("project", 8, "fp32")
    knots = b.knots().cpu().numpy()
    vals = b.values().cpu().numpy()
    off = b.offsets()
    for i, f in enumerate(funcs):
        kn = knots[off[i]:off[i + 1]]
        vref = oracle.values(f, kn, "project")
        assert np.abs(vals[off[i]:off[i + 1]] - vref).max() <= 2.5 * fp32_integrand_envelope(f), i
    b.close()


@pytest.mark.parametrize("F", [40, 70])
def test_batch_fp32_projection_of_a_constant_is_exact(pwl, F):
    # a constant is exact in FP32 and in the CPWL space (the hats sum to one),
    # so P_T gives it back at every vertex: what remains is the error of the
    # float-float hat sums and of the FP64 solve, far below FP32 rounding
    c = 0.7503662109375  # 2^-1 + ... : exact in FP32
    funcs = [{"kind": "poly", "a": -3.0 + 0.01 * k, "b": 2.0 + 0.37 * k, "p": [c, 0, 0, 0, 0, 0, 0, 0]}
             for k in range(F)]
    n_int = [1 + (37 * k) % 900 for k in range(F)]
    b = pwl.Batch(funcs, n_int, m_per_interval=4)
    b.design()
    b.project("project", 8, "fp32")
    vals = b.values().cpu().numpy()
    assert np.abs(vals - c).max() <= 1e-12 * c
    b.close()


@pytest.mark.parametrize("cells_per_knot", [1, 4])
def test_batch_staged_and_direct_pieces_agree(pwl, workloads, cells_per_knot):
    # staging only changes where the records are read from: the results of
    # every plan (never / default / always staged) and every CTA shape are
    # bit-identical and match the oracle; one cell per knot makes cells that
    # hold several knots (chain walks)
    funcs, n_int, qo, x = _batch_inputs(workloads, 30, seed=12)
    b = pwl.Batch(funcs, n_int, m_per_interval=8, cells_per_knot=cells_per_knot)
    b.design()
    b.project("project")
    b.build()
    xd = torch.tensor(x, device="cuda")
    outs = []
    for shape in range(5):
        for stage_min in (0, 16, 1 << 30):
            b.plan(qo, shape, stage_min)
            info = b.info()
            if stage_min == 0:
                assert info["n_staged"] == 0
            if stage_min == 1 << 30:
                assert info["n_staged"] == 0 if shape == 3 else info["n_staged"] > 0
            outs.append(b.eval(xd).cpu().numpy())
    b.check()  # no staging wait timed out
    for o in outs[1:]:
        assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32))
    _check_batch_eval(b, funcs, qo, x, outs[0])
    b.close()


@pytest.mark.parametrize("stage_min", [1, 16, 1 << 30])
def test_batch_many_functions_per_cta(pwl, workloads, stage_min):
    # 600 functions for ~150 CTAs: every CTA walks several functions, so the
    # asynchronous path (shape 4) alternates its two record buffers and
    # prefetches across staged and unstaged pieces
    funcs, n_int, qo, x = _batch_inputs(workloads, 600, seed=17, knots_hi=300, q_hi=2e4)
    b = pwl.Batch(funcs, n_int, m_per_interval=4)
    b.design()
    b.project("project")
    b.build()
    xd = torch.tensor(x, device="cuda")
    b.plan(qo, 4, stage_min)  # the asynchronous (bulk copy) shape
    info = b.info()
    assert info["n_items"] > info["eval_grid"]
    y = b.eval(xd).cpu().numpy()
    b.check()
    _check_batch_eval(b, funcs, qo, x, y)
    b.plan(qo, 3)
    y3 = b.eval(xd).cpu().numpy()
    assert np.array_equal(y.view(np.uint32), y3.view(np.uint32))
    b.close()


def test_batch_plan_covers_every_query_once(pwl, workloads):
    # y pre-filled with a sentinel: every planned query is written, the
    # spare element after the last one is not
    funcs, n_int, qo, x = _batch_inputs(workloads, 25, seed=13, q_hi=4e5)
    b = pwl.Batch(funcs, n_int, m_per_interval=8)
    b.design()
    b.project("interp")
    b.build()
    m = int(qo[-1])
    xd = torch.tensor(np.r_[x, np.float32(0.5)], device="cuda")
    y = torch.full((m + 1,), float("inf"), device="cuda")
    b.plan(qo)
    info = b.info()
    assert info["total_queries"] == m and info["n_items"] >= 1
    b.eval(xd[:m], y[:m])
    yh = y.cpu().numpy()
    assert np.isinf(yh[m])
    assert not np.isinf(yh[:m]).any()
    _check_batch_eval(b, funcs, qo, x, yh[:m])
    b.close()


def test_batch_autotune_keeps_results(pwl, workloads):
    funcs, n_int, qo, x = _batch_inputs(workloads, 20, seed=14)
    b = pwl.Batch(funcs, n_int, m_per_interval=8)
    b.design()
    b.project("project")
    b.build()
    xd = torch.tensor(x, device="cuda")
    b.plan(qo)
    ref = b.eval(xd).cpu().numpy()
    y = torch.empty_like(xd)
    b.autotune(xd, y, reps=1)
    info = b.info()
    assert 0 <= info["eval_shape"] < 5 and info["stage_min"] in (0, 4, 16, 64)
    b.check()  # no staging wait timed out
    got = b.eval(xd).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    b.close()


def test_batch_fp32_density_design(pwl, workloads):
    funcs, n_int, _, _ = _batch_inputs(workloads, 12, seed=15)
    b = pwl.Batch(funcs, n_int, m_per_interval=32)
    b.design("fp32")
    knots = b.knots().cpu().numpy()
    off = b.offsets()
    for i, f in enumerate(funcs):
        ref = oracle.design(f, n_int[i], 32 * n_int[i])
        assert np.all(np.abs(knots[off[i]:off[i + 1]] - ref) <= fp32_design_bound(ref)), i
    b.close()


def test_batch_fp64_bessel_large_arguments(pwl):
    # J0(alpha x) on [0, 50] with alpha up to 5: z = alpha x up to 250, where
    # the FP64 J0/J1 must stay near 1e-16 for the knots to meet DESIGN_REL
    funcs = [{"kind": "bessel_j0", "a": 0.0, "b": 50.0, "p": [1.0, al]} for al in (3.0, 4.2, 5.0, 0.7)]
    n_int = [2500, 4000, 3100, 4095]
    b = pwl.Batch(funcs, n_int, m_per_interval=16)
    b.design("fp64")
    b.project("project")
    knots = b.knots().cpu().numpy()
    vals = b.values().cpu().numpy()
    off = b.offsets()
    for i, f in enumerate(funcs):
        kn = knots[off[i]:off[i + 1]]
        ref = oracle.design(f, n_int[i], 16 * n_int[i])
        assert np.abs(kn - ref).max() <= DESIGN_REL * (f["b"] - f["a"]), i
        vref = oracle.values(f, kn, "project")
        assert np.abs(vals[off[i]:off[i + 1]] - vref).max() <= VALUES_REL * np.abs(vref).max(), i
    b.close()


def test_batch_design_degenerate_densities(pwl):
    # f linear (f'' = 0): G_M = 0 and the uniform partition, as the oracle;
    # a Gaussian on [-30, 30] in FP32 mode: the FP32 density underflows to 0
    # over long stretches at both ends (chunks without a cell of positive
    # density), while the knots, set by the mass in the middle, stay within
    # the FP32-mode tolerance of the FP64 oracle
    lin = {"kind": "poly", "a": -1.0, "b": 2.0, "p": [3.0, -0.5]}
    wide = {"kind": "gaussian", "a": -30.0, "b": 30.0, "p": [1.0, 0.0, 1.0]}
    funcs = [lin, wide, lin, wide]
    n_int = [12, 200, 1, 33]
    for prec in ("fp64", "fp32"):
        b = pwl.Batch(funcs, n_int, m_per_interval=64)
        b.design(prec)
        kn = b.knots().cpu().numpy()
        off = b.offsets()
        for i, f in enumerate(funcs):
            got = kn[off[i]:off[i + 1]]
            ref = oracle.design(f, n_int[i], 64 * n_int[i])
            if f is lin:
                assert np.allclose(got, -1.0 + np.arange(n_int[i] + 1) * 3.0 / n_int[i], atol=1e-15)
            elif prec == "fp64":
                assert np.abs(got - ref).max() <= DESIGN_REL * (f["b"] - f["a"])
            else:
                assert np.all(np.abs(got - ref) <= fp32_design_bound(ref))
            assert np.all(np.diff(got) > 0)
        b.close()


def test_batch_pipeline_in_a_cuda_graph(pwl, workloads):
    # design, projection, index build and evaluation enqueue no host
    # synchronisation and allocate nothing: captured once, replayed, they
    # give the eager results bit for bit
    funcs, n_int, qo, x = _batch_inputs(workloads, 16, seed=16)
    b = pwl.Batch(funcs, n_int, m_per_interval=16)
    xd = torch.tensor(x, device="cuda")
    b.design("fp32")
    b.project("project", precision="fp32")
    b.build()
    b.plan(qo)
    eager = b.eval(xd).cpu().numpy()
    y = torch.zeros_like(xd)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            b.design("fp32", stream=s)
            b.project("project", precision="fp32", stream=s)
            b.build(stream=s)
            b.eval(xd, y, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        y.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(y.cpu().numpy().view(np.uint32), eager.view(np.uint32))
    b.close()


def test_batch_check_flags_bad_knots(pwl):
    funcs = [{"kind": "gaussian", "a": -4.0, "b": 4.0, "p": [1.0, 0.0, 1.0]}] * 3
    b = pwl.Batch(funcs, [8, 8, 8], m_per_interval=4)
    b.design()
    b.project("interp")
    b.build()
    b.check()
    kv = b.knots(copy=False)
    kv[9 + 4] = kv[9 + 3]  # function 1: a repeated knot
    b.build()
    with pytest.raises(pwl.PwlError, match="function 1"):
        b.check()
    b.close()


def test_batch_rejects_bad_arguments(pwl):
    g = {"kind": "gaussian", "a": -4.0, "b": 4.0, "p": [1.0, 0.0, 1.0]}
    with pytest.raises(pwl.PwlError):
        pwl.Batch([g, g], [8, 0])
    with pytest.raises(pwl.PwlError):
        pwl.Batch([g], [70000])
    with pytest.raises(pwl.PwlError):
        pwl.Batch([dict(g, a=1.0, b=1.0)], [8])
    b = pwl.Batch([g, g], [8, 9])
    b.design()
    b.project("interp")
    b.build()
    x = torch.zeros(17, device="cuda")
    with pytest.raises(pwl.PwlError, match="plan"):
        b.eval(x)
    with pytest.raises(pwl.PwlError):
        b.plan([0, 5, 3])
    with pytest.raises(pwl.PwlError):
        b.plan([1, 5, 9])
    with pytest.raises(pwl.PwlError):
        b.plan([0, 5, 9], shape=7)
    b.plan([0, 8, 16])
    with pytest.raises(ValueError):
        b.eval(x[:15])
    with pytest.raises(pwl.PwlError, match="aligned"):
        b.eval(x[1:])
    b.plan([0, 0, 0])
    b.eval(x[:0])  # no queries: a no-op
    b.close()
