"""GPU parity of the paper's comparison paths (Section V, Table I) through
the C ABI, against the FP64 oracle:

- direct evaluation of f (pwl_direct_eval): expf and the SFU's __expf for
  the Gaussian, IEEE and fast division for the Lorentzian, the math
  library's j0f and the one-term asymptotic J0 (Section V-C), each within
  the error bound of its FP32 arithmetic and of the CUDA functions'
  documented accuracy;
- the CPWL evaluation variants that mirror Table I's rows: the paper's
  branch-free unrolled binary search (mode 0), search + texture filter
  (mode 4), the uniform-partition texture lookup (mode 5);
- the register-generated (compute-ceiling) form of each, whose checksum is
  recomputed on the host from the same counter-based query generator.
"""
import numpy as np
import pytest

import oracle
from pwl_testutil import EVAL_REL, round_knots, round_values

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS = 2.0**-24  # unit roundoff of FP32


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


GAUSS = [{"kind": "gaussian", "a": -4.0, "b": 4.0, "p": [1.0, 0.0, 1.0]},
         {"kind": "gaussian", "a": -3.0, "b": 5.0, "p": [0.7, 0.4, 1.7]}]
LORENTZ = [{"kind": "lorentzian", "a": -10.0, "b": 10.0, "p": [1.0, 0.0, 1.0]},
           {"kind": "lorentzian", "a": -2.0, "b": 6.0, "p": [1.0 / np.pi, 0.5, 0.3]}]
J0 = [{"kind": "bessel_j0", "a": 0.0, "b": 50.0, "p": [1.0, 1.0]},
      {"kind": "bessel_j0", "a": 0.0, "b": 20.0, "p": [0.5, 2.3]}]


def direct_bound(desc, method, x):
    """Per-query bound on |GPU - f(x)| for pwl_direct_eval (x: the FP32
    queries widened to FP64), from the FP32 roundings of the parameters and
    of each operation, plus the documented accuracy of the CUDA functions:
    expf 2 ulp, __expf 2 + floor(1.173 |t|) ulp at argument t, IEEE division
    0.5 ulp, __fdividef 2 ulp, j0f 9 ulp below 8 and 2.2e-6 absolute above."""
    A, c, d = desc["p"][0], desc["p"][1], desc["p"][2] if len(desc["p"]) > 2 else 0.0
    fx = np.abs(oracle.f_many(desc, x))
    if desc["kind"] == "gaussian":
        u = (x - c) / d
        t = 0.5 * u * u
        # u: rounding of mu, of x - mu, of 1/s and of the product; t adds
        # one more; the result two (times A, A rounded)
        du = EPS * (3 * np.abs(u) + abs(c) / d)
        dt = np.abs(u) * du + EPS * t
        lib = 4 * EPS if method == "library" else 2 * EPS * (2 + np.floor(1.173 * t))
        return fx * (dt + lib + 3 * EPS) + 1e-38
    if desc["kind"] == "lorentzian":
        u = (x - c) / d
        du = EPS * (3 * np.abs(u) + abs(c) / d)
        dden = (2 * np.abs(u) * du + EPS * (1 + u * u)) / (1 + u * u)
        lib = EPS if method == "library" else 4 * EPS
        return fx * (dden + lib + 2 * EPS) + 1e-38
    # J0(alpha x): z = alpha x carries two roundings (alpha, product)
    sc = pytest.importorskip("scipy.special")
    z = c * x
    dz = 2 * EPS * np.abs(z)
    j0 = np.abs(sc.j0(z))
    lib = np.where(np.abs(z) < 8, 9 * 2 * EPS * j0, 2.2e-6)
    return abs(A) * (lib + np.abs(sc.j1(z)) * dz + 2 * EPS * j0) + 1e-38


def one_term_bound(desc, x):
    """|GPU - oracle one-term form| for the asymptotic J0 (z >= 1): the
    phase z - pi/4 carries the roundings of z (2 eps z) and of the
    subtraction, and the SFU cosine's argument reduction adds about as much
    again (its absolute error is 2^-21.41 on [-pi, pi]); rsqrtf 2 ulp and
    the amplitude's rounding act on sqrt(2/(pi z))."""
    A, alpha = desc["p"][0], desc["p"][1]
    z = alpha * x
    s = np.sqrt(2.0 / (np.pi * z))
    return abs(A) * s * (2.0**-21.41 + 8 * EPS * np.abs(z) + 8 * EPS) + 1e-38


@pytest.mark.parametrize("method", ["library", "fast"])
@pytest.mark.parametrize("desc", GAUSS + LORENTZ + J0, ids=lambda d: d["kind"])
def test_direct_eval_matches_oracle(pwl, workloads, desc, method):
    m = (1 << 20) + 3
    x = workloads.uniform_queries(desc, m, seed=21)
    x[:5] = torch.tensor([desc["a"], desc["b"], 0.5 * (desc["a"] + desc["b"]), desc["b"], desc["a"]],
                         device="cuda")
    y = pwl.pwl_direct_eval(desc, method, x).cpu().numpy().astype(np.float64)
    xs = x.cpu().numpy().astype(np.float64)
    if desc["kind"] == "bessel_j0" and method == "fast":
        keep = desc["p"][1] * xs >= 1.0  # the expansion is for z >> 1/4
        ref = oracle.j0_one_term(desc, xs[keep])
        assert np.all(np.abs(y[keep] - ref) <= one_term_bound(desc, xs[keep]))
        return
    ref = oracle.f_many(desc, xs)
    err = np.abs(y - ref)
    assert np.all(err <= direct_bound(desc, method, xs)), float(np.max(err / direct_bound(desc, method, xs)))


def test_direct_eval_alignment_in_place_and_sizes(pwl, workloads):
    desc = GAUSS[0]
    base = workloads.uniform_queries(desc, 4099, seed=3)
    xs = base.cpu().numpy().astype(np.float64)
    ref = oracle.f_many(desc, xs)
    bnd = direct_bound(desc, "library", xs)
    buf = torch.empty(4099 + 8, device="cuda")
    for off in (0, 1, 2, 3):
        for m in (0, 1, 5, 4096 - off):
            x = buf[off:off + m]  # views at 4-byte offsets: scalar heads and tails
            x.copy_(base[:m])
            y = pwl.pwl_direct_eval(desc, "library", x)
            if m:
                assert np.all(np.abs(y.cpu().numpy() - ref[:m]) <= bnd[:m])
    x = base.clone()
    pwl.pwl_direct_eval(desc, "library", x, x)  # y = x
    assert np.all(np.abs(x.cpu().numpy() - ref) <= bnd)
    with pytest.raises(pwl.PwlError):
        pwl.pwl_direct_eval({"kind": "poly", "a": 0.0, "b": 1.0, "p": [1.0]}, "library", base)


@pytest.mark.parametrize("method", ["library", "fast"])
@pytest.mark.parametrize("desc", [GAUSS[0], LORENTZ[0], {"kind": "bessel_j0", "a": 1.0, "b": 50.0, "p": [1.0, 1.0]}],
                         ids=lambda d: d["kind"])
def test_direct_synthetic_checksum_matches_oracle(pwl, workloads, desc, method):
    # the generated queries are rebuilt on the host from the published hash;
    # the GPU sums every thread's share in FP32
    m, seed = (1 << 20) + 5, 777
    got = pwl.pwl_direct_synthetic(desc, method, m, seed).item()
    x = workloads.synthetic_queries(desc["a"], desc["b"], m, seed).astype(np.float64)
    if desc["kind"] == "bessel_j0" and method == "fast":
        ref_y, bnd = oracle.j0_one_term(desc, x), one_term_bound(desc, x)
    else:
        ref_y, bnd = oracle.f_many(desc, x), direct_bound(desc, method, x)
    ref = float(np.sum(ref_y))
    assert abs(got - ref) <= float(np.sum(bnd)) + 1e-5 * float(np.sum(np.abs(ref_y)))


# ---- CPWL evaluation variants of Table I -----------------------------------------
def _table(pwl, f, N, uniform=False):
    if uniform:
        kn = torch.tensor(f["a"] + (f["b"] - f["a"]) * np.arange(N + 1) / N, dtype=torch.float64, device="cuda")
        kn[-1] = f["b"]
    else:
        kn = pwl.pwl_design(f, N)
    vals = pwl.pwl_project(f, kn, "interp")
    t = pwl.Table(kn, vals)
    return t, round_knots(kn.cpu().numpy()), round_values(vals.cpu().numpy(), "fp32")


def _edge_queries(workloads, f, xk, m, seed):
    x = workloads.uniform_queries(f, m, seed=seed)
    n = min(len(xk), m // 4)
    x[:n] = torch.tensor(xk[:n], dtype=torch.float32, device="cuda")
    x[n:n + 4] = torch.tensor([f["a"] - 1.0, f["b"] + 1.0, float("nan"), float("inf")], device="cuda")
    return x


def _tex_bound(xk, vk, xs):
    # 8 fractional bits of texture weight: |v_i - v_{i-1}| / 256, taken over
    # the query's interval and its neighbours (a coordinate within an ulp
    # of a knot may round to the next texel)
    i = np.clip(np.searchsorted(xk, xs, side="right"), 1, len(xk) - 1)
    dv = np.abs(np.diff(vk))
    dvn = np.maximum(dv[i - 1], np.maximum(dv[np.maximum(i - 2, 0)], dv[np.minimum(i, len(dv) - 1)]))
    return dvn / 256.0 + 1e-6 * np.abs(vk).max()


@pytest.mark.parametrize("N", [1, 2, 31, 255, 1023, 4096, 16383])
def test_search_variant_matches_oracle(pwl, workloads, N):
    # mode 0: Algorithm 1 with the unrolled branch-free search (Section IV)
    f = workloads.PAPER_FUNCTIONS["bessel_j0"]
    t, xk, vk = _table(pwl, f, N)
    x = _edge_queries(workloads, f, xk, (1 << 18) + 3, seed=5)
    y = t.variant(0, x).cpu().numpy().astype(np.float64)
    ref = oracle.evaluate(xk, vk, x.cpu().numpy().astype(np.float64))
    nan = np.isnan(ref)
    assert np.array_equal(nan, np.isnan(y))
    assert np.abs(y[~nan] - ref[~nan]).max() <= EVAL_REL * np.abs(ref[~nan]).max()
    t.close()


def test_search_variant_rejects_tables_beyond_its_unrolled_size(pwl, workloads):
    f = workloads.PAPER_FUNCTIONS["gaussian"]
    t, _, _ = _table(pwl, f, 16384)
    x = workloads.uniform_queries(f, 1000, seed=1)
    for mode in (0, 4):
        with pytest.raises(pwl.PwlError, match="NOTSUP|search path"):
            t.variant(mode, x)
    t.close()


@pytest.mark.parametrize("N", [1, 63, 1024, 4096])
def test_search_texture_variant_matches_oracle(pwl, workloads, N):
    # mode 4: the search of mode 0, then the texture filter
    for name in ("gaussian", "lorentzian"):
        f = workloads.PAPER_FUNCTIONS[name]
        t, xk, vk = _table(pwl, f, N)
        x = _edge_queries(workloads, f, xk, (1 << 18) + 1, seed=6)
        y = t.variant(4, x).cpu().numpy().astype(np.float64)
        xs = x.cpu().numpy().astype(np.float64)
        ref = oracle.evaluate(xk, vk, xs)
        nan = np.isnan(ref)
        assert np.array_equal(nan, np.isnan(y))
        assert np.all(np.abs(y[~nan] - ref[~nan]) <= _tex_bound(xk, vk, xs[~nan]))
        t.close()


@pytest.mark.parametrize("N", [1, 64, 1024, 4096])
def test_uniform_texture_variant_matches_oracle(pwl, workloads, N):
    # mode 5: uniform partition, texture coordinate straight from x (no search)
    f = workloads.PAPER_FUNCTIONS["gaussian"]
    t, xk, vk = _table(pwl, f, N, uniform=True)
    x = _edge_queries(workloads, f, xk, (1 << 18) + 1, seed=7)
    y = t.variant(5, x).cpu().numpy().astype(np.float64)
    xs = x.cpu().numpy().astype(np.float64)
    ref = oracle.evaluate(xk, vk, xs)
    nan = np.isnan(ref)
    assert np.array_equal(nan, np.isnan(y))
    # the coordinate (x - x_0) N / (x_N - x_0) also carries a few FP32
    # roundings of size eps N: tiny against the 1/256 of the weight
    assert np.all(np.abs(y[~nan] - ref[~nan]) <= 1.01 * _tex_bound(xk, vk, xs[~nan]))
    t.close()


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4, 5, 6])
def test_synthetic_variant_checksums_match_oracle(pwl, workloads, mode):
    f = workloads.PAPER_FUNCTIONS["lorentzian"]
    t, xk, vk = _table(pwl, f, 1000, uniform=(mode == 5))
    m, seed = (1 << 20) + 9, 4242
    got = pwl.pwl_eval_synthetic_variant(t.handle, mode, m, seed).item()
    x = workloads.synthetic_queries(float(t.info["a"]), float(t.info["b"]), m, seed).astype(np.float64)
    ref_y = oracle.evaluate(xk, vk, x)
    ref = float(np.sum(ref_y))
    per = _tex_bound(xk, vk, x) if mode in (1, 4, 5) else EVAL_REL * np.abs(vk).max()
    bound = float(np.sum(per)) + 1e-5 * float(np.sum(np.abs(ref_y)))
    assert abs(got - ref) <= bound
    t.close()
