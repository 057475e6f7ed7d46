"""GPU vs oracle parity of the channel-wise map (one CPWL function per
channel, Algorithm 1 per element) and its backward, through the C ABI."""
import numpy as np
import pytest

import oracle
from pwl_testutil import EVAL_REL, GRAD_REL

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pwl():
    import paper_1510_02975_gb300 as m
    from paper_1510_02975_gb300 import _build
    _build.build()
    return m


def _channel_tables(pwl, C, N, seed=0):
    """Gaussian-designed knots on [-8, 8] and P_T values, perturbed per
    channel by small seeded noise (the learnable-map initialisation)."""
    f = {"kind": "gaussian", "a": -8.0, "b": 8.0, "p": [1.0, 0.0, 1.0]}
    k = pwl.pwl_design(f, N).cpu().numpy()
    v = pwl.pwl_project(f, pwl.pwl_design(f, N), "project").cpu().numpy()
    rng = np.random.default_rng(seed)
    h = np.diff(k).min()
    knots = np.tile(k, (C, 1))
    knots[:, 1:-1] += rng.uniform(-0.2, 0.2, (C, N - 1)) * h
    values = np.tile(v, (C, 1)) + rng.normal(scale=1e-3, size=(C, N + 1))
    return knots.astype(np.float32), values.astype(np.float32)


def _oracle_rows(knots, values, x):
    C = knots.shape[0]
    out = np.empty(x.shape, np.float64)
    for c in range(C):
        out[:, c] = oracle.evaluate(knots[c].astype(np.float64), values[c].astype(np.float64), x[:, c])
    return out


@pytest.mark.parametrize("C,N,R", [(16, 256, 4099), (40, 256, 3000), (7, 31, 1000), (33, 1, 500)])
def test_channels_forward_matches_oracle(pwl, C, N, R):
    knots, values = _channel_tables(pwl, C, N)
    g = torch.Generator(device="cuda").manual_seed(4)
    x = torch.randn(R, C, generator=g, device="cuda") * 2.0
    x[0, :] = float("nan")
    x[1, :] = 9.0
    x[2, :] = -9.0
    x[3, :] = torch.tensor(knots[:, N // 2], device="cuda")
    kt = torch.tensor(knots, device="cuda")
    vt = torch.tensor(values, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = pwl.pwl_channels_forward(kt, vt, x, status=st)
    assert int(st.item()) == 0
    ref = _oracle_rows(knots, values, x.cpu().numpy().astype(np.float64))
    got = y.cpu().numpy().astype(np.float64)
    assert np.array_equal(np.isnan(ref), np.isnan(got))
    ok = ~np.isnan(ref)
    assert np.abs(got[ok] - ref[ok]).max() <= EVAL_REL * np.abs(ref[ok]).max()


@pytest.mark.parametrize("k_cells", [3, 40, 300])
def test_channels_forward_with_chains(pwl, k_cells):
    C, N, R = 20, 256, 2000
    knots, values = _channel_tables(pwl, C, N, seed=1)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(R, C, generator=g, device="cuda") * 2.0
    y = pwl.pwl_channels_forward(torch.tensor(knots, device="cuda"), torch.tensor(values, device="cuda"), x,
                                 k_cells=k_cells)
    ref = _oracle_rows(knots, values, x.cpu().numpy().astype(np.float64))
    assert np.abs(y.cpu().numpy() - ref).max() <= EVAL_REL * np.abs(ref).max()


def test_channels_forward_bf16_io(pwl):
    C, N, R = 48, 256, 3001
    knots, values = _channel_tables(pwl, C, N, seed=2)
    g = torch.Generator(device="cuda").manual_seed(6)
    x = (torch.randn(R, C, generator=g, device="cuda") * 2.0).to(torch.bfloat16)
    y = pwl.pwl_channels_forward(torch.tensor(knots, device="cuda"), torch.tensor(values, device="cuda"), x)
    ref = _oracle_rows(knots, values, x.float().cpu().numpy().astype(np.float64))
    got = y.float().cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 2.0**-8 * np.abs(ref) * 1.0001 + EVAL_REL * np.abs(ref).max())


@pytest.mark.parametrize("io", ["fp32", "bf16"])
def test_channels_forward_aligned_and_unaligned_x_agree(pwl, io):
    # the same x at a 16-byte aligned base and at a base 2 or 4 bytes off:
    # the same y bit for bit, and the oracle's values on a partial last tile
    # (44 channels: 4 past the last full 8-channel tile), ragged rows (5003),
    # NaN, clamped and at-knot queries.
    C, N, R = 44, 256, 5003
    knots, values = _channel_tables(pwl, C, N, seed=7)
    g = torch.Generator(device="cuda").manual_seed(9)
    x = torch.randn(R, C, generator=g, device="cuda") * 2.0
    x[0, :] = float("nan")
    x[1, :] = 9.0
    x[2, :] = -9.0
    x[3, :] = torch.tensor(knots[:, N // 3], device="cuda")
    if io == "bf16":
        x = x.to(torch.bfloat16)
    kt, vt = torch.tensor(knots, device="cuda"), torch.tensor(values, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    y1 = pwl.pwl_channels_forward(kt, vt, x, status=st)
    buf = torch.empty(R * C + 1, dtype=x.dtype, device="cuda")
    xu = buf[1:].view(R, C)
    xu.copy_(x)
    assert xu.data_ptr() % 16 != 0
    y2 = pwl.pwl_channels_forward(kt, vt, xu, status=st)
    assert int(st.item()) == 0
    assert torch.equal(torch.isnan(y1), torch.isnan(y2))
    assert torch.equal(torch.nan_to_num(y1), torch.nan_to_num(y2))
    ref = _oracle_rows(knots, values, x.float().cpu().numpy().astype(np.float64))
    got = y1.float().cpu().numpy().astype(np.float64)
    assert np.array_equal(np.isnan(ref), np.isnan(got))
    ok = ~np.isnan(ref)
    if io == "fp32":
        assert np.abs(got[ok] - ref[ok]).max() <= EVAL_REL * np.abs(ref[ok]).max()
    else:
        assert np.all(np.abs(got[ok] - ref[ok]) <= 2.0**-8 * np.abs(ref[ok]) * 1.0001 + EVAL_REL * np.abs(ref[ok]).max())


def test_channels_non_increasing_knots_flagged(pwl):
    C, N = 16, 8
    knots = np.tile(np.linspace(-1, 1, N + 1), (C, 1)).astype(np.float32)
    knots[5, 3] = knots[5, 2]
    values = np.zeros_like(knots)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    pwl.pwl_channels_forward(torch.tensor(knots, device="cuda"), torch.tensor(values, device="cuda"),
                             torch.zeros(10, C, device="cuda"), status=st)
    assert int(st.item()) & 1


@pytest.mark.parametrize("C,N,R,k_cells", [(16, 256, 4096, 0), (37, 64, 3001, 0), (20, 256, 2000, 50)])
def test_channels_backward_matches_oracle(pwl, C, N, R, k_cells):
    knots, values = _channel_tables(pwl, C, N, seed=3)
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(R, C, generator=g, device="cuda") * 2.0
    x[0, :] = -9.0
    x[1, :] = 9.0
    x[2, :] = torch.tensor(knots[:, 0], device="cuda")
    x[3, :] = torch.tensor(knots[:, N], device="cuda")
    x[4, :] = torch.tensor(knots[:, N // 3], device="cuda")
    gy = torch.randn(R, C, generator=g, device="cuda")
    gv = torch.zeros(C, N + 1, device="cuda")
    gk = torch.zeros(C, N + 1, device="cuda")
    kt, vt = torch.tensor(knots, device="cuda"), torch.tensor(values, device="cuda")
    gx = pwl.pwl_channels_backward(kt, vt, x, gy, None, gv, gk, k_cells=k_cells)
    xs = x.cpu().numpy().astype(np.float64)
    gys = gy.cpu().numpy().astype(np.float64)
    gxg, gvg, gkg = gx.cpu().numpy(), gv.cpu().numpy(), gk.cpu().numpy()
    for c in range(C):
        rgx, rgv, rgk, rva, rka = oracle.evaluate_grad(knots[c].astype(np.float64), values[c].astype(np.float64),
                                                       xs[:, c], gys[:, c])
        assert np.abs(gxg[:, c] - rgx).max() <= EVAL_REL * max(np.abs(rgx).max(), 1e-30)
        assert np.all(np.abs(gvg[c] - rgv) <= GRAD_REL * rva + 1e-30)
        assert np.all(np.abs(gkg[c] - rgk) <= GRAD_REL * rka + 1e-30)


def test_channel_autograd_matches_finite_differences(pwl):
    # d/d(values, knots) of sum(w * y) by central differences in FP64 on the
    # oracle, compared with the autograd gradients of the GPU map
    C, N, R = 3, 6, 64
    rng = np.random.default_rng(8)
    base = np.linspace(-2, 2, N + 1)
    knots = np.tile(base, (C, 1)) + np.c_[np.zeros(C), rng.uniform(-0.1, 0.1, (C, N - 1)), np.zeros(C)]
    values = rng.normal(size=(C, N + 1))
    x = rng.uniform(-2.5, 2.5, (R, C))
    w = rng.normal(size=(R, C))
    kt = torch.tensor(knots, dtype=torch.float32, device="cuda", requires_grad=True)
    vt = torch.tensor(values, dtype=torch.float32, device="cuda", requires_grad=True)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    y = pwl.ChannelPWL.apply(xt, kt, vt)
    (y * torch.tensor(w, dtype=torch.float32, device="cuda")).sum().backward()
    k32 = kt.detach().cpu().numpy().astype(np.float64)
    v32 = vt.detach().cpu().numpy().astype(np.float64)
    x32 = xt.detach().cpu().numpy().astype(np.float64)

    def loss(kk, vv):
        return sum(np.dot(w[:, c], oracle.evaluate(kk[c], vv[c], x32[:, c])) for c in range(C))

    eps = 1e-6
    for c in range(C):
        for j in range(N + 1):
            dv = np.zeros_like(v32)
            dv[c, j] = eps
            fd_v = (loss(k32, v32 + dv) - loss(k32, v32 - dv)) / (2 * eps)
            assert abs(vt.grad[c, j].item() - fd_v) <= 1e-4 * max(1.0, abs(fd_v))
            if 0 < j < N:
                fd_k = (loss(k32 + dv, v32) - loss(k32 - dv, v32)) / (2 * eps)
                assert abs(kt.grad[c, j].item() - fd_k) <= 1e-3 * max(1.0, abs(fd_k))


def test_channel_autograd_bf16_input(pwl):
    # a BF16 map differentiates too: gx comes back in BF16, and the gradients
    # equal the FP32 backward's on the widened inputs (BF16 -> FP32 is exact)
    C, N, R = 24, 64, 2001
    knots, values = _channel_tables(pwl, C, N, seed=9)
    g = torch.Generator(device="cuda").manual_seed(10)
    x16 = (torch.randn(R, C, generator=g, device="cuda") * 2.0).to(torch.bfloat16).requires_grad_(True)
    gy = torch.randn(R, C, generator=g, device="cuda").to(torch.bfloat16)
    kt = torch.tensor(knots, device="cuda", requires_grad=True)
    vt = torch.tensor(values, device="cuda", requires_grad=True)
    st = pwl.ChannelPWL.new_status()
    y = pwl.ChannelPWL.apply(x16, kt, vt, status=st)
    assert y.dtype == torch.bfloat16
    y.backward(gy)
    pwl.ChannelPWL.check(st)
    assert x16.grad.dtype == torch.bfloat16
    gv = torch.zeros(C, N + 1, device="cuda")
    gk = torch.zeros(C, N + 1, device="cuda")
    gx = pwl.pwl_channels_backward(kt.detach(), vt.detach(), x16.detach().float(), gy.float(), None, gv, gk)
    assert torch.equal(x16.grad, gx.to(torch.bfloat16))
    xs = x16.detach().float().cpu().numpy().astype(np.float64)
    gys = gy.float().cpu().numpy().astype(np.float64)
    for c in range(C):
        _, rgv, rgk, rva, rka = oracle.evaluate_grad(knots[c].astype(np.float64), values[c].astype(np.float64),
                                                     xs[:, c], gys[:, c])
        assert np.all(np.abs(vt.grad[c].cpu().numpy() - rgv) <= GRAD_REL * rva + 1e-30)
        assert np.all(np.abs(kt.grad[c].cpu().numpy() - rgk) <= GRAD_REL * rka + 1e-30)


def test_channel_autograd_reports_crossed_knots(pwl):
    # a training step that makes two knots of a channel cross is visible to
    # the caller through the status word of the autograd path
    C, N, R = 16, 32, 256
    knots, values = _channel_tables(pwl, C, N, seed=11)
    knots[7, 10], knots[7, 11] = knots[7, 11], knots[7, 10]
    kt = torch.tensor(knots, device="cuda", requires_grad=True)
    vt = torch.tensor(values, device="cuda", requires_grad=True)
    x = torch.zeros(R, C, device="cuda", requires_grad=True)
    st = pwl.ChannelPWL.new_status()
    pwl.ChannelPWL.apply(x, kt, vt, status=st).sum().backward()
    with pytest.raises(pwl.PwlError, match="not strictly increasing"):
        pwl.ChannelPWL.check(st)
    st.zero_()
    ok = pwl.ChannelPWL.new_status()
    pwl.ChannelPWL.apply(x, torch.tensor(_channel_tables(pwl, C, N, seed=11)[0], device="cuda"), vt, status=ok)
    pwl.ChannelPWL.check(ok)
