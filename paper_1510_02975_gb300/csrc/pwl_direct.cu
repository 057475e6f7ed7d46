// pwl_direct.cu -- direct evaluation of f, the comparison systems of the
// paper's timings (Section V): the Gaussian with the C library's expf and
// with the SFU's __expf (Table I), the Lorentzian with an IEEE division and
// with the fast division (Section V-B), and J0 with the CUDA library's j0f
// and with the first term of its asymptotic expansion evaluated by the SFU's
// cosine and reciprocal square root (Section V-C):
//     J0(z) ~ sqrt(2 / (pi z)) cos(z - pi/4),   z >> 1/4.
//
// Each runs in the streaming shape of pwl_eval (16-byte vectors, several
// loads in flight per thread, persistent grid), so that the two can be
// compared at the same bytes per query, and on register-generated queries
// (the compute ceiling, no memory traffic), where the paper's synthetic
// comparison lives.
#include <math.h>

#include "pwl_stream.cuh"

namespace pwl {

namespace {

// FP32 constants of one function, formed in FP64 on the host and rounded:
//   Gaussian   A exp(-((x - mu)/s)^2 / 2):  {A, mu, 1/s}
//   Lorentzian A / (1 + ((x - x0)/g)^2):    {A, x0, 1/g}
//   J0         A J0(alpha x):               {A, alpha, A sqrt(2/pi)}
struct DirectParams {
    float A, c, d;
};

// METHOD 0: the library functions (expf, IEEE division, j0f); METHOD 1: the
// fast forms (__expf, __fdividef, the asymptotic J0 with __cosf and rsqrtf).
template <int KIND, int METHOD>
struct Direct {
    DirectParams q;
    __device__ __forceinline__ float operator()(float x) const
    {
        if constexpr (KIND == PWL_F_GAUSSIAN) {
            const float u = (x - q.c) * q.d;
            const float e = -0.5f * u * u;
            return q.A * (METHOD == 0 ? expf(e) : __expf(e));
        } else if constexpr (KIND == PWL_F_LORENTZIAN) {
            const float u = (x - q.c) * q.d;
            const float den = __fmaf_rn(u, u, 1.0f);
            return METHOD == 0 ? __fdiv_rn(q.A, den) : __fdividef(q.A, den);
        } else {
            const float z = q.c * x;
            if constexpr (METHOD == 0) {
                return q.A * j0f(z);
            } else {
                // pi/4 rounded to FP32
                return q.d * rsqrtf(z) * __cosf(z - 0.785398163397448f);
            }
        }
    }
};

struct DirectIO {
    const float* x;
    float* y;
    int64_t m, head, nvec;
    uint32_t seed;
    double* sum;
    float a, b;  // generated queries: x_q = u_q (b - a) + a
};

constexpr int kDirectUnroll = 4;

template <int KIND, int METHOD, bool SYNTH>
__global__ void __launch_bounds__(1024) direct_kernel(const DirectParams q, const DirectIO io)
{
    __shared__ float s_red[32];
    const Direct<KIND, METHOD> f{q};
    if constexpr (SYNTH)
        cta_sum_to(synth_sum(f, io.seed, io.a, __fsub_rn(io.b, io.a), io.m), s_red, io.sum);
    else
        stream_body<float, kDirectUnroll>(io.head, io.nvec, f, io.x, io.y, io.m);
}

using DirectKern = void (*)(const DirectParams, const DirectIO);

template <bool SYNTH>
DirectKern pick(int kind, int method)
{
    switch (kind * 2 + method) {
    case PWL_F_GAUSSIAN * 2 + 0: return direct_kernel<PWL_F_GAUSSIAN, 0, SYNTH>;
    case PWL_F_GAUSSIAN * 2 + 1: return direct_kernel<PWL_F_GAUSSIAN, 1, SYNTH>;
    case PWL_F_LORENTZIAN * 2 + 0: return direct_kernel<PWL_F_LORENTZIAN, 0, SYNTH>;
    case PWL_F_LORENTZIAN * 2 + 1: return direct_kernel<PWL_F_LORENTZIAN, 1, SYNTH>;
    case PWL_F_BESSEL_J0 * 2 + 0: return direct_kernel<PWL_F_BESSEL_J0, 0, SYNTH>;
    case PWL_F_BESSEL_J0 * 2 + 1: return direct_kernel<PWL_F_BESSEL_J0, 1, SYNTH>;
    }
    return nullptr;
}

pwl_status direct_setup(const pwl_func* f, int32_t method, DirectParams* q)
{
    if (!f) return fail(PWL_EINVAL, "f is NULL");
    pwl_status st = validate_func(f);
    if (st != PWL_OK) return st;
    if (method != 0 && method != 1) return fail(PWL_EINVAL, "method must be 0 (library) or 1 (fast)");
    switch (f->kind) {
    case PWL_F_GAUSSIAN:
    case PWL_F_LORENTZIAN:
        *q = DirectParams{(float)f->p[0], (float)f->p[1], (float)(1.0 / f->p[2])};
        return PWL_OK;
    case PWL_F_BESSEL_J0:
        *q = DirectParams{(float)f->p[0], (float)f->p[1], (float)(f->p[0] * sqrt(2.0 / M_PI))};
        return PWL_OK;
    }
    return fail(PWL_ENOTSUP, "direct evaluation covers the Gaussian, Lorentzian and J0 kinds (got kind %d)",
                f->kind);
}

pwl_status direct_launch(DirectKern kern, const DirectParams& q, const DirectIO& io, int64_t units, cudaStream_t s)
{
    int max_grid = 0;
    PWL_CUDA_TRY(occupancy_grid_fn(reinterpret_cast<const void*>(kern), 1024, 0, &max_grid));
    kern<<<stream_grid(max_grid, units, 1024, kDirectUnroll), 1024, 0, s>>>(q, io);
    PWL_CHECK_LAUNCH("direct_kernel");
    return PWL_OK;
}

}  // namespace

}  // namespace pwl

using namespace pwl;

extern "C" {

pwl_status pwl_direct_eval(const pwl_func* f, int32_t method, const float* d_x, float* d_y, int64_t m, void* stream)
{
    clear_error();
    DirectParams q;
    pwl_status st = direct_setup(f, method, &q);
    if (st != PWL_OK) return st;
    if (m < 0) return fail(PWL_EINVAL, "m must be >= 0");
    if (m > 0 && (!d_x || !d_y)) return fail(PWL_EINVAL, "x / y is NULL");
    if (m == 0) return PWL_OK;
    DirectIO io{};
    io.x = d_x;
    io.y = d_y;
    io.m = m;
    stream_split<float>(d_x, d_y, m, &io.head, &io.nvec);
    return direct_launch(pick<false>(f->kind, method), q, io, io.nvec + (m - io.nvec * 4), as_stream(stream));
}

pwl_status pwl_direct_synthetic(const pwl_func* f, int32_t method, uint32_t seed, int64_t m, double* d_sum,
                                void* stream)
{
    clear_error();
    DirectParams q;
    pwl_status st = direct_setup(f, method, &q);
    if (st != PWL_OK) return st;
    if (m < 0 || m > ((int64_t)1 << 32)) return fail(PWL_EINVAL, "m must be in [0, 2^32]");
    if (!d_sum) return fail(PWL_EINVAL, "d_sum is NULL");
    if (m == 0) return PWL_OK;
    DirectIO io{};
    io.m = m;
    io.seed = seed;
    io.sum = d_sum;
    io.a = (float)f->a;
    io.b = (float)f->b;
    return direct_launch(pick<true>(f->kind, method), q, io, (m + 3) / 4, as_stream(stream));
}

}  // extern "C"
