"""The allocation-free backward entry point, pwl_eval_backward_noalloc.

Callers that cannot allocate device memory while they run (real-time loops
with memory fixed at start-up, code called back from a host framework that
owns the device memory, callers with no workspace to lend) use this variant:
it keeps its per-CTA partial sums in the library's static device array
instead of a caller workspace.  Its results must match pwl_eval_backward's on
the same inputs, on two calls in a row (the second sees the array as the
first left it).  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from pwl_testutil import GRAD_REL, round_knots, round_values

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def env():
    import paper_1510_02975_gb300 as pwl
    from paper_1510_02975_gb300 import _build, _capi
    from paper_1510_02975_gb300 import workloads as W
    _build.build()
    return pwl, _capi.load(), W


@pytest.mark.parametrize("name,N", [("lorentzian", 1024), ("bessel_j0", 4096), ("gaussian", 5)])
def test_noalloc_backward_matches_workspace_backward(env, name, N):
    pwl, lib, W = env
    f = W.PAPER_FUNCTIONS[name]
    knots = pwl.pwl_design(f, N)
    vals = pwl.pwl_project(f, knots, "project")
    table = pwl.Table(knots, vals)
    m = (1 << 20) + 5
    x = W.uniform_queries(f, m, seed=11)
    x[:64] = float(f["a"]) - 1.0  # clamped queries too
    gy = W.upstream_grad((m,), seed=12)

    # the existing entry point, with a caller workspace
    gx_ref = torch.empty_like(x)
    gv_ref = torch.zeros(N + 1, device="cuda")
    gk_ref = torch.zeros(N + 1, device="cuda")
    pwl.pwl_eval_backward(table.handle, x, gy, gx_ref, gv_ref, gk_ref)

    # tolerance of the table gradients: GRAD_REL of the sum of |terms|
    _, _, _, gva, gka = oracle.evaluate_grad(round_knots(knots.cpu().numpy()), round_values(vals.cpu().numpy(), "fp32"),
                                             x.cpu().numpy().astype(np.float64), gy.cpu().numpy().astype(np.float64))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        gx = torch.full_like(x, float("nan"))
        gv = torch.zeros(N + 1, device="cuda")
        gk = torch.zeros(N + 1, device="cuda")
        st = lib.pwl_eval_backward_noalloc(ctypes.c_void_p(table.handle), _p(x), _p(gy), _p(gx), _p(gv), _p(gk), m,
                                           stream)
        assert st == 0, lib.pwl_last_error()
        torch.cuda.synchronize()
        assert torch.equal(gx, gx_ref)
        assert np.all(np.abs((gv - gv_ref).cpu().numpy()) <= GRAD_REL * gva + 1e-30)
        assert np.all(np.abs((gk - gk_ref).cpu().numpy()) <= GRAD_REL * gka + 1e-30)
    table.close()


def test_noalloc_backward_rejects_tables_beyond_the_static_scratch(env):
    pwl, lib, W = env
    f = W.GAUSSIAN
    N = 8000  # 2 (N + 2) floats per SM no longer fit 2^21 floats on a 152-SM GPU
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if 2 * (N + 2) * sms <= (1 << 21):
        pytest.skip("GPU with few SMs: N = 8000 still fits")
    knots = pwl.pwl_design(f, N)
    table = pwl.Table(knots, pwl.pwl_project(f, knots, "interp"))
    x = W.uniform_queries(f, 1000, seed=1)
    gy = torch.ones_like(x)
    gx = torch.empty_like(x)
    st = lib.pwl_eval_backward_noalloc(ctypes.c_void_p(table.handle), _p(x), _p(gy), _p(gx), None, None, x.numel(),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 1  # PWL_EINVAL
    assert b"static scratch" in lib.pwl_last_error()
    table.close()
