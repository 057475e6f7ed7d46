// pwl_errors.cu -- a priori L2 errors of the CPWL approximations and the N
// that reaches a target error (Results 4-6, Section III-B):
//   interpolant on the nearly optimal partition T*:
//       ||f - pi_T* f|| ~ (int |f''|^{2/5})^{5/2} / (N^2 sqrt(120)),
//   orthogonal projection: ||f - P_T f|| ~ ||f - pi_T f|| / sqrt(6) (the
//       per-interval ratio h^5/720 : h^5/120 of Results 2-3, any partition),
//   interpolant on the uniform partition:
//       ||f - pi_U f|| ~ (b - a)^2 ||f''|| / (N^2 sqrt(120)).
// The two integrals come from the midpoint rule on the design's cells
// (t_k = a + (k + 1/2) delta, FP64), the same discretisation pwl_design uses
// for the knot density.
#include <math.h>

#include <algorithm>

#include "pwl_design.cuh"

namespace pwl {

namespace {

constexpr int kConstThreads = 256;

// out[0] += delta * sum_k |f''(t_k)|^{2/5}, out[1] += delta * sum_k f''(t_k)^2
template <bool SAMPLED>
__global__ void __launch_bounds__(kConstThreads) error_constants_kernel(pwl_func F, int64_t M, double* out)
{
    __shared__ double s_red[2][kConstThreads / 32];
    const double delta = (F.b - F.a) / (double)M;
    double s25 = 0.0, s2 = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < M; k += stride) {
        const double t = __dadd_rn(F.a, __dmul_rn((double)k + 0.5, delta));
        const double f2 = func_second_derivative_k<SAMPLED, double>(F, t);
        s25 += pow_two_fifths(f2);
        s2 = __fma_rn(f2, f2, s2);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s25 += __shfl_xor_sync(0xffffffffu, s25, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_red[0][warp] = s25;
        s_red[1][warp] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kConstThreads / 32; ++w) {
            a += s_red[0][w];
            b += s_red[1][w];
        }
        atomicAdd(out, a * delta);
        atomicAdd(out + 1, b * delta);
    }
}

// C / N^2 with C the error constant of (form, partition)
double error_constant(double int_f2_25, double int_f2_sq, double a, double b, int32_t form, int32_t uniform)
{
    const double c = uniform ? (b - a) * (b - a) * sqrt(int_f2_sq) : pow(int_f2_25, 2.5);
    return c / sqrt(120.0) / (form == PWL_PROJECT ? sqrt(6.0) : 1.0);
}

pwl_status check_error_args(double int_f2_25, double int_f2_sq, double a, double b, int32_t form)
{
    if (!(int_f2_25 >= 0.0) || !(int_f2_sq >= 0.0) || !isfinite(int_f2_25) || !isfinite(int_f2_sq))
        return fail(PWL_EINVAL, "the integrals must be finite and >= 0");
    if (!isfinite(a) || !isfinite(b) || !(a < b)) return fail(PWL_EINVAL, "need finite a < b");
    if (form != PWL_INTERP && form != PWL_PROJECT) return fail(PWL_EINVAL, "unknown form %d", form);
    return PWL_OK;
}

}  // namespace

}  // namespace pwl

using namespace pwl;

extern "C" {

pwl_status pwl_error_constants(const pwl_func* f, int64_t m_cells, double* d_out, void* stream)
{
    clear_error();
    pwl_status st = validate_func(f);
    if (st != PWL_OK) return st;
    if (!d_out) return fail(PWL_EINVAL, "d_out is NULL");
    if (m_cells < 0) return fail(PWL_EINVAL, "m_cells must be >= 0");
    const int64_t M = m_cells > 0 ? m_cells : ((int64_t)1 << 20);
    cudaStream_t s = as_stream(stream);
    PWL_CUDA_TRY(cudaMemsetAsync(d_out, 0, 2 * sizeof(double), s));
    const int64_t blocks = std::min<int64_t>((M + kConstThreads - 1) / kConstThreads, (int64_t)device_info().sms * 8);
    if (f->kind == PWL_F_SAMPLED)
        error_constants_kernel<true><<<(int)blocks, kConstThreads, 0, s>>>(*f, M, d_out);
    else
        error_constants_kernel<false><<<(int)blocks, kConstThreads, 0, s>>>(*f, M, d_out);
    PWL_CHECK_LAUNCH("error_constants_kernel");
    return PWL_OK;
}

pwl_status pwl_predicted_error(double int_f2_25, double int_f2_sq, double a, double b, int64_t n_intervals,
                               int32_t form, int32_t uniform, double* err_out)
{
    clear_error();
    if (!err_out) return fail(PWL_EINVAL, "err_out is NULL");
    if (n_intervals < 1) return fail(PWL_EINVAL, "n_intervals must be >= 1");
    pwl_status st = check_error_args(int_f2_25, int_f2_sq, a, b, form);
    if (st != PWL_OK) return st;
    const double n = (double)n_intervals;
    *err_out = error_constant(int_f2_25, int_f2_sq, a, b, form, uniform) / (n * n);
    return PWL_OK;
}

pwl_status pwl_n_for_error(double int_f2_25, double int_f2_sq, double a, double b, double target_l2, int32_t form,
                           int32_t uniform, int64_t* n_out)
{
    clear_error();
    if (!n_out) return fail(PWL_EINVAL, "n_out is NULL");
    if (!(target_l2 > 0.0) || !isfinite(target_l2)) return fail(PWL_EINVAL, "target_l2 must be finite and > 0");
    pwl_status st = check_error_args(int_f2_25, int_f2_sq, a, b, form);
    if (st != PWL_OK) return st;
    const double c = error_constant(int_f2_25, int_f2_sq, a, b, form, uniform);
    // smallest N >= 1 with c / N^2 <= target
    double n = ceil(sqrt(c / target_l2));
    if (!(n <= (double)kMaxIntervals)) return fail(PWL_EINVAL, "the target needs more than %d intervals", kMaxIntervals);
    int64_t N = std::max<int64_t>(1, (int64_t)n);
    while (N > 1 && c / ((double)(N - 1) * (double)(N - 1)) <= target_l2) --N;
    while (c / ((double)N * (double)N) > target_l2) ++N;
    *n_out = N;
    return PWL_OK;
}

}  // extern "C"
