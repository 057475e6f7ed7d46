"""GPU vs oracle parity at the benchmark's full sizes, in the launch
configurations bench.py times: 2^28 queries per table (Algorithm 1 and its
backward), the channel-wise map on x[65536, 4096] with 257 knots per channel,
and the 4096-function batch.  Outputs the oracle can compute one by one are
compared on samples (random indices, the first and last rows or queries, and
whole channels or functions); sums over every query are checked through
identities that hold at any size:
  - the hat weights of a query sum to one (1 - delta + delta, or 1 at a
    clamped end), so sum_j g_v[j] = sum_q gy_q;
  - y depends on x and the knots only through x - x_{i-1} and x_i - x_{i-1}
    (translation invariance), so dy/dx + sum_k dy/dx_k = 0 and
    sum_k g_k[k] = -sum_q g_x[q]."""
import numpy as np
import pytest

import oracle
from pwl_testutil import EVAL_REL, GRAD_REL, fp32_design_bound, round_knots, round_values

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M_FULL = 1 << 28
ROWS, CHANNELS, CH_N = 65536, 4096, 256


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


@pytest.fixture(autouse=True)
def _release_memory():
    yield
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _sample_indices(m, n_random=1 << 16, edge=2048, seed=0):
    rng = np.random.default_rng(seed)
    idx = np.concatenate([rng.integers(0, m, n_random), np.arange(min(edge, m)), np.arange(max(m - edge, 0), m)])
    return np.unique(idx)


def _table(pwl, f, N, form="project"):
    knots = pwl.pwl_design(f, N)
    vals = pwl.pwl_project(f, knots, form)
    t = pwl.Table(knots, vals)
    return t, round_knots(knots.cpu().numpy()), round_values(vals.cpu().numpy(), "fp32")


@pytest.mark.parametrize("name,N", [("gaussian", 256), ("lorentzian", 1024), ("bessel_j0", 4096)])
def test_eval_full_size_sampled(pwl, workloads, name, N):
    f = workloads.PAPER_FUNCTIONS[name]
    t, xk, vk = _table(pwl, f, N)
    idx = torch.tensor(_sample_indices(M_FULL), device="cuda")
    for make, seed in ((workloads.uniform_queries, 1), (workloads.normal_queries, 2)):
        x = make(f, M_FULL, seed=seed)
        y = torch.empty_like(x)
        pwl.pwl_eval(t.handle, x, y)
        xs = x[idx].cpu().numpy().astype(np.float64)
        got = y[idx].cpu().numpy().astype(np.float64)
        ref = oracle.evaluate(xk, vk, xs)
        assert np.abs(got - ref).max() <= EVAL_REL * np.abs(ref).max()
        assert bool(torch.isfinite(y).all())
        del x, y
    t.close()


@pytest.mark.parametrize("name,N", [("gaussian", 256), ("lorentzian", 4096)])
def test_backward_full_size_sampled_and_sums(pwl, workloads, name, N):
    f = workloads.PAPER_FUNCTIONS[name]
    t, xk, vk = _table(pwl, f, N)
    x = workloads.uniform_queries(f, M_FULL, seed=1)
    gy = workloads.upstream_grad((M_FULL,), seed=5)
    gv = torch.zeros(N + 1, device="cuda")
    gk = torch.zeros(N + 1, device="cuda")
    gx = pwl.pwl_eval_backward(t.handle, x, gy, None, gv, gk)
    idx = torch.tensor(_sample_indices(M_FULL, seed=1), device="cuda")
    rgx = oracle.evaluate_grad(xk, vk, x[idx].cpu().numpy().astype(np.float64),
                               gy[idx].cpu().numpy().astype(np.float64))[0]
    assert np.abs(gx[idx].cpu().numpy() - rgx).max() <= EVAL_REL * np.abs(rgx).max()
    sum_gy = float(gy.double().sum())
    abs_gy = float(gy.double().abs().sum())
    sum_gx = float(gx.double().sum())
    abs_gx = float(gx.double().abs().sum())
    assert abs(float(gv.double().sum()) - sum_gy) <= GRAD_REL * abs_gy
    assert abs(float(gk.double().sum()) + sum_gx) <= GRAD_REL * abs_gx
    t.close()


def _bench_channel_tables(pwl):
    """The channel tables of the benchmark: the Gaussian design and P_T values
    on [-8, 8] with 257 knots, replicated, knots jittered by +-0.2 h_min and
    values by N(0, 1e-3) per channel (CUDA generator, seed 4)."""
    f = {"kind": "gaussian", "a": -8.0, "b": 8.0, "p": [1.0, 0.0, 1.0]}
    k64 = pwl.pwl_design(f, CH_N)
    v64 = pwl.pwl_project(f, k64, "project")
    g = torch.Generator(device="cuda").manual_seed(4)
    h = float(torch.diff(k64).min())
    knots = k64.float().repeat(CHANNELS, 1)
    knots[:, 1:-1] += (torch.rand(CHANNELS, CH_N - 1, generator=g, device="cuda") - 0.5) * 0.4 * h
    values = v64.float().repeat(CHANNELS, 1) + torch.randn(CHANNELS, CH_N + 1, generator=g, device="cuda") * 1e-3
    return knots, values


def _sample_channels(seed=0, n=24):
    rng = np.random.default_rng(seed)
    fixed = [0, 1, 7, 8, 31, 32, 33, 127, 128, 2047, 2048, 4064, 4095]
    return np.unique(np.concatenate([fixed, rng.integers(0, CHANNELS, n)]))


def test_channels_forward_full_size_sampled(pwl, workloads):
    knots, values = _bench_channel_tables(pwl)
    x = workloads.channel_inputs(ROWS, CHANNELS, seed=4)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = pwl.pwl_channels_forward(knots, values, x, status=st)
    assert int(st.item()) == 0
    kn, vv = knots.cpu().numpy().astype(np.float64), values.cpu().numpy().astype(np.float64)
    cs = _sample_channels()
    xs = x[:, cs].cpu().numpy().astype(np.float64)
    ys = y[:, cs].cpu().numpy().astype(np.float64)
    for j, c in enumerate(cs):  # every row of the sampled channels
        ref = oracle.evaluate(kn[c], vv[c], xs[:, j])
        assert np.abs(ys[:, j] - ref).max() <= EVAL_REL * np.abs(ref).max(), c
    # BF16 I/O on the same rows: one BF16 rounding of the FP32-accurate value
    xb = x.to(torch.bfloat16)
    del x, y
    yb = pwl.pwl_channels_forward(knots, values, xb, status=st)
    assert int(st.item()) == 0
    xbs = xb[:, cs].float().cpu().numpy().astype(np.float64)
    ybs = yb[:, cs].float().cpu().numpy().astype(np.float64)
    for j, c in enumerate(cs):
        ref = oracle.evaluate(kn[c], vv[c], xbs[:, j])
        assert np.all(np.abs(ybs[:, j] - ref) <= 2.0**-8 * np.abs(ref) * 1.0001 + EVAL_REL * np.abs(ref).max()), c


def test_channels_backward_full_size(pwl, workloads):
    knots, values = _bench_channel_tables(pwl)
    x = workloads.channel_inputs(ROWS, CHANNELS, seed=4)
    gy = workloads.upstream_grad((ROWS, CHANNELS), seed=5)
    gv = torch.zeros_like(values)
    gk = torch.zeros_like(knots)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    gx = pwl.pwl_channels_backward(knots, values, x, gy, None, gv, gk, status=st)
    assert int(st.item()) == 0
    # every channel: the two identities over its 65536 rows (clamped rows add
    # gy to an end value and nothing to the knots, which both sums respect)
    sum_gy, abs_gy = gy.double().sum(0), gy.double().abs().sum(0)
    sum_gx, abs_gx = gx.double().sum(0), gx.double().abs().sum(0)
    assert bool(((gv.double().sum(1) - sum_gy).abs() <= GRAD_REL * abs_gy).all())
    assert bool(((gk.double().sum(1) + sum_gx).abs() <= GRAD_REL * abs_gx + 1e-30).all())
    # sampled channels: the oracle's gradients over all of their rows
    kn, vv = knots.cpu().numpy().astype(np.float64), values.cpu().numpy().astype(np.float64)
    cs = _sample_channels(seed=1, n=16)
    xs = x[:, cs].cpu().numpy().astype(np.float64)
    gys = gy[:, cs].cpu().numpy().astype(np.float64)
    gxs = gx[:, cs].cpu().numpy()
    gvs, gks = gv[cs].cpu().numpy(), gk[cs].cpu().numpy()
    for j, c in enumerate(cs):
        rgx, rgv, rgk, rva, rka = oracle.evaluate_grad(kn[c], vv[c], xs[:, j], gys[:, j])
        assert np.abs(gxs[:, j] - rgx).max() <= EVAL_REL * max(np.abs(rgx).max(), 1e-30), c
        assert np.all(np.abs(gvs[j] - rgv) <= GRAD_REL * rva + 1e-30), c
        assert np.all(np.abs(gks[j] - rgk) <= GRAD_REL * rka + 1e-30), c


def test_batch_full_size_sampled(pwl, workloads):
    # the benchmark's batch: 4096 functions, FP32-density design with 16
    # density cells per interval, P_T values, the autotuned evaluation
    funcs, n_int, n_q = workloads.batch_functions(4096, seed=3)
    x, qo = workloads.batch_queries(funcs, n_q, seed=6)
    y = torch.empty_like(x)
    b = pwl.Batch(funcs, n_int, m_per_interval=16)
    b.design("fp32")
    b.project("project", 8, "fp32")
    b.build()
    b.check()
    b.plan(qo)
    b.autotune(x, y, reps=1)
    y.fill_(float("nan"))
    b.eval(x, y)
    knots = b.knots().cpu().numpy()
    xk = b.knots_fp32().cpu().numpy().astype(np.float64)
    vk = b.values_fp32().cpu().numpy().astype(np.float64)
    off = b.offsets()
    rng = np.random.default_rng(0)
    fs = np.unique(np.concatenate([[0, 1, 2, len(funcs) - 1], rng.integers(0, len(funcs), 40)]))
    for i in fs:
        f = funcs[i]
        kn = knots[off[i]:off[i + 1]]
        ref = oracle.design(f, n_int[i], 16 * n_int[i])
        assert np.all(np.abs(kn - ref) <= fp32_design_bound(ref)), i
        q0, q1 = int(qo[i]), int(qo[i + 1])
        xs = x[q0:q1].cpu().numpy().astype(np.float64)
        got = y[q0:q1].cpu().numpy().astype(np.float64)
        vv = vk[off[i]:off[i + 1]]
        r = oracle.evaluate(xk[off[i]:off[i + 1]], vv, xs)
        assert np.abs(got - r).max() <= EVAL_REL * np.abs(vv).max(), i
    assert bool(torch.isfinite(y).all())  # every query written
    b.close()
