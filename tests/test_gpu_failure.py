"""Failure detection on the GPU without a fault (the error paths of the
library, driven by its injection hooks):

- allocation failures: every call that allocates device memory returns
  PWL_ENOMEM, releases what it had taken, leaves existing state usable, and
  works again once allocations succeed;
- the bounded waits of the asynchronous batch evaluation: with an arrival
  withheld from every staging barrier, each wait runs out after a short
  limit, the kernel retires cleanly (its copies landed, the context stays
  usable), pwl_batch_check reports PWL_ETIMEOUT once, and the next
  evaluation is correct again."""
import numpy as np
import pytest

import oracle
from pwl_testutil import EVAL_REL, round_knots, round_values

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PWL_ENOMEM, PWL_ETIMEOUT = 2, 5


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


@pytest.fixture
def alloc_hook(pwl):
    yield pwl.pwl_test_fail_allocations
    pwl.pwl_test_fail_allocations(-1)


@pytest.mark.parametrize("succeed_first", [0, 1])
def test_table_build_enomem_at_each_allocation(pwl, workloads, alloc_hook, succeed_first):
    f = workloads.GAUSSIAN
    kn = pwl.pwl_design(f, 256)
    v = pwl.pwl_project(f, kn, "project")
    alloc_hook(succeed_first)  # 0: the table's base allocation fails; 1: its records
    with pytest.raises(pwl.PwlError) as ei:
        pwl.Table(kn, v)
    assert ei.value.status == PWL_ENOMEM
    alloc_hook(-1)
    t = pwl.Table(kn, v)
    x = workloads.uniform_queries(f, 100003, seed=1)
    ref = oracle.evaluate(round_knots(kn.cpu().numpy()), round_values(v.cpu().numpy(), "fp32"),
                          x.cpu().numpy().astype(np.float64))
    assert np.abs(t(x).cpu().numpy() - ref).max() <= EVAL_REL * np.abs(ref).max()
    t.close()


def test_texture_enomem_leaves_the_table_usable(pwl, workloads, alloc_hook):
    f = workloads.LORENTZIAN
    kn = pwl.pwl_design(f, 512)
    v = pwl.pwl_project(f, kn, "interp")
    t = pwl.Table(kn, v)
    x = workloads.uniform_queries(f, 65537, seed=2)
    alloc_hook(0)
    with pytest.raises(pwl.PwlError) as ei:
        t.variant(1, x)
    assert ei.value.status == PWL_ENOMEM
    y_main = t(x)  # the main path allocates nothing
    alloc_hook(-1)
    xk, vk = round_knots(kn.cpu().numpy()), round_values(v.cpu().numpy(), "fp32")
    xs = x.cpu().numpy().astype(np.float64)
    ref = oracle.evaluate(xk, vk, xs)
    assert np.abs(y_main.cpu().numpy() - ref).max() <= EVAL_REL * np.abs(ref).max()
    y_tex = t.variant(1, x).cpu().numpy().astype(np.float64)  # the texture is created now
    i = np.clip(np.searchsorted(xk, xs, side="right"), 1, len(xk) - 1)
    assert np.all(np.abs(y_tex - ref) <= np.abs(vk[i] - vk[i - 1]) / 256.0 + 1e-6 * np.abs(vk).max())
    t.close()


def _small_batch(pwl, workloads, F=24, seed=5):
    funcs, n_int, n_q = workloads.batch_functions(F, seed=seed, knots_lo=16, knots_hi=600, q_lo=2e3, q_hi=5e4)
    rng = np.random.default_rng(seed)
    xs = [rng.uniform(f["a"], f["b"], nq).astype(np.float32) for f, nq in zip(funcs, n_q)]
    qo = np.concatenate([[0], np.cumsum(n_q)]).astype(np.int64)
    x = np.concatenate(xs)
    b = pwl.Batch(funcs, n_int, m_per_interval=16)
    b.design()
    b.project("project")
    b.build()
    b.check()
    return b, funcs, qo, x


def _check_batch(b, funcs, qo, x, y):
    xk = b.knots_fp32().cpu().numpy().astype(np.float64)
    vk = b.values_fp32().cpu().numpy().astype(np.float64)
    off = b.offsets()
    for f in range(len(funcs)):
        q0, q1 = int(qo[f]), int(qo[f + 1])
        if q1 > q0:
            ref = oracle.evaluate(xk[off[f]:off[f + 1]], vk[off[f]:off[f + 1]], x[q0:q1].astype(np.float64))
            assert np.abs(y[q0:q1] - ref).max() <= EVAL_REL * np.abs(vk[off[f]:off[f + 1]]).max(), f


def test_batch_create_and_plan_enomem(pwl, workloads, alloc_hook):
    funcs, n_int, n_q = workloads.batch_functions(8, seed=2, knots_lo=16, knots_hi=300, q_lo=100, q_hi=1000)
    alloc_hook(0)
    with pytest.raises(pwl.PwlError) as ei:
        pwl.Batch(funcs, n_int)
    assert ei.value.status == PWL_ENOMEM
    alloc_hook(-1)
    b, funcs, qo, x = _small_batch(pwl, workloads)
    xd = torch.tensor(x, device="cuda")
    b.plan(qo, shape=0)
    alloc_hook(0)
    with pytest.raises(pwl.PwlError) as ei:
        b.plan(qo, shape=2)  # a new plan needs an allocation: the old one stays
    assert ei.value.status == PWL_ENOMEM
    y = b.eval(xd)
    alloc_hook(-1)
    _check_batch(b, funcs, qo, x, y.cpu().numpy().astype(np.float64))
    b.close()


def test_batch_async_wait_timeout_is_reported_and_recovered(pwl, workloads):
    b, funcs, qo, x = _small_batch(pwl, workloads)
    xd = torch.tensor(x, device="cuda")
    b.plan(qo, shape=4, stage_min=64)  # the asynchronous shape, every piece staged
    assert b.info()["n_staged"] > 0
    y = b.eval(xd)
    b.check()
    _check_batch(b, funcs, qo, x, y.cpu().numpy().astype(np.float64))
    # every staging wait now runs out after 2 ms
    pwl.pwl_batch_inject_wait_timeout(b.handle, True, 2_000_000)
    y2 = torch.full_like(xd, float("nan"))
    b.eval(xd, y2)
    torch.cuda.synchronize()  # the launch retired: no wait outlived its limit
    with pytest.raises(pwl.PwlError) as ei:
        b.check()
    assert ei.value.status == PWL_ETIMEOUT
    assert torch.isnan(y2).any()  # the CTAs stopped before their staged pieces
    b.check()  # the check cleared the flag
    pwl.pwl_batch_inject_wait_timeout(b.handle, False, 0)
    y3 = b.eval(xd)
    b.check()
    _check_batch(b, funcs, qo, x, y3.cpu().numpy().astype(np.float64))
    b.close()
