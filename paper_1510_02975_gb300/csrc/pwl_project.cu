// pwl_project.cu -- vertex values of the two CPWL approximations of
// Section II-B: the interpolant pi_T f (v_i = f(x_i), Eq. 3) and the L2
// orthogonal projection P_T f (Eqs. 4-6).
//
// P_T: one thread per interval computes the two hat-weighted integrals
// int f phi_{j-1} and int f phi_j over I_j by Q-point Gauss-Legendre (FP64
// sums; f in FP64 or FP32); then one CTA per function assembles the
// tridiagonal Gram system (M_ii = (h_i + h_{i+1})/3, M_{i,i+1} = h_{i+1}/6,
// b_i = R_i + L_{i+1}) in shared memory and solves it in FP64 by cyclic
// reduction: log2(N) levels of independent row eliminations instead of the
// O(N) dependent chain of the Thomas algorithm the paper names, which on a
// GPU with few FP64 units per SM would be latency bound.
#include <math.h>

#include <algorithm>

#include <mutex>

#include "pwl_design.cuh"

namespace pwl {

namespace {

constexpr int kSolveThreads = 1024;

// index f with koff[f] - f <= g < koff[f+1] - (f+1): the function owning
// global interval g (intervals of f start at koff[f] - f).
__device__ __forceinline__ int find_interval_owner(const int64_t* __restrict__ koff, int F, int64_t g)
{
    int lo = 0, hi = F - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(koff + mid) - mid <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_knot_owner(const int64_t* __restrict__ koff, int F, int64_t g)
{
    int lo = 0, hi = F - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(koff + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void interp_values_kernel(ProjectPlan p)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < p.total_knots; g += stride) {
        const int f = find_knot_owner(p.koff, p.F, g);
        p.values[g] = (double)func_value<T>(p.funcs[f], (T)p.knots[g]);
    }
}

// (L_j, R_j) = (int_{I_j} f phi_{j-1}, int_{I_j} f phi_j) for every interval.
// At the node t_q = mid + half x_q the hats are phi_{j-1} = (1 - x_q)/2 and
// phi_j = (1 + x_q)/2, so L_j = half sum_q wl_q f(t_q) and
// R_j = half sum_q wr_q f(t_q) with the host-side weights wl, wr: no
// division per node.  FP64 mode: t_q and the sums in FP64.  FP32 mode: t_q
// and f(t_q) in FP32 (the argument of an FP32 f is rounded to FP32 anyway),
// the sums in FP64.
template <typename T>
__global__ void hat_integrals_kernel(ProjectPlan p, const __grid_constant__ GaussLegendre gl)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < p.total_intervals;
         g += stride) {
        const int f = find_interval_owner(p.koff, p.F, g);
        const int64_t j = g - (p.koff[f] - f) + 1;  // interval index 1..N_f
        const double* x = p.knots + p.koff[f];
        const double xl = x[j - 1], xr = x[j];
        const double mid = 0.5 * (xl + xr), half = 0.5 * (xr - xl);
        const pwl_func F = p.funcs[f];
        double L = 0.0, R = 0.0;
        if constexpr (sizeof(T) == 4) {
            const float midf = (float)mid, halff = (float)half;
            for (int q = 0; q < gl.Q; ++q) {
                const double fv = (double)func_value<float>(F, __fmaf_rn(halff, gl.xf[q], midf));
                L = __fma_rn(gl.wl[q], fv, L);
                R = __fma_rn(gl.wr[q], fv, R);
            }
        } else {
            for (int q = 0; q < gl.Q; ++q) {
                const double fv = func_value<double>(F, __fma_rn(half, gl.x[q], mid));
                L = __fma_rn(gl.wl[q], fv, L);
                R = __fma_rn(gl.wr[q], fv, R);
            }
        }
        p.lr[g] = make_double2(half * L, half * R);
    }
}

// Gram system of a batch of functions, one thread per function: the
// Thomas algorithm (forward elimination, back substitution) in FP64, the
// rows assembled on the fly (M_{i,i-1} = h_i/6, M_ii = (h_i + h_{i+1})/3,
// M_{i,i+1} = h_{i+1}/6, b_i = R_i + L_{i+1}).  O(N) operations per
// function and no barriers: the right solver when thousands of functions
// run at once; the forward multipliers go to scratch, the values array
// holds the eliminated right-hand side until back substitution.
__global__ void gram_thomas_kernel(ProjectPlan p)
{
    const int stride = gridDim.x * blockDim.x;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < p.F; f += stride) {
        const int64_t k0 = p.koff[f];
        const int n = (int)(p.koff[f + 1] - k0);
        const int N = n - 1;
        const double* x = p.knots + k0;
        const double2* lr = p.lr + (k0 - f);
        double* cp = p.cr + 4 * k0;  // forward multipliers c'_i
        double* dv = p.values + k0;  // d'_i, then the solution
        constexpr double kSixth = 1.0 / 6.0, kThird = 1.0 / 3.0;
        double xm = x[0], x0 = x[0], x1 = N >= 1 ? x[1] : x[0];
        double cprev = 0.0, dprev = 0.0;
        double2 lprev = make_double2(0.0, 0.0);
        for (int i = 0; i < n; ++i) {
            const double hl = i > 0 ? x0 - xm : 0.0;
            const double hr = i < N ? x1 - x0 : 0.0;
            const double2 lri = i < N ? lr[i] : make_double2(0.0, 0.0);
            const double rhs = lprev.y + lri.x;
            const double lower = hl * kSixth;
            const double denom = (hl + hr) * kThird - lower * cprev;
            const double r = 1.0 / denom;
            cprev = (i < N) ? hr * kSixth * r : 0.0;
            dprev = (rhs - lower * dprev) * r;
            cp[i] = cprev;
            dv[i] = dprev;
            lprev = lri;
            xm = x0;
            x0 = x1;
            x1 = (i + 2 <= N) ? x[i + 2] : x1;
        }
        double v = dv[N];
        for (int i = N - 1; i >= 0; --i) {
            v = dv[i] - cp[i] * v;
            dv[i] = v;
        }
    }
}

// Gram system of the hat basis and its solution by cyclic reduction.  Rows
// 0..n-1 (n = N+1).  Forward: for strides s = 1, 2, 4, ... while 2s-1 < n,
// every row i = 2s-1 (mod 2s) eliminates its couplings to rows i-s and i+s
// (coefficients a: to i-s, c: to i+s).  One row (s_top - 1) is then
// uncoupled; back substitution fills rows s-1 (mod 2s) for s = s_top/2..1.
__global__ void __launch_bounds__(kSolveThreads) gram_solve_kernel(ProjectPlan p, int use_smem)
{
    extern __shared__ double s_cr[];
    for (int f = blockIdx.x; f < p.F; f += gridDim.x) {
        const int64_t k0 = p.koff[f];
        const int n = (int)(p.koff[f + 1] - k0);
        const int N = n - 1;
        const double* x = p.knots + k0;
        const double2* lr = p.lr + (k0 - f);
        double* A;
        if (use_smem) A = s_cr; else A = p.cr + 4 * k0;
        double* B = A + n;
        double* C = B + n;
        double* D = C + n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const double hl = (i > 0) ? x[i] - x[i - 1] : 0.0;
            const double hr = (i < N) ? x[i + 1] - x[i] : 0.0;
            A[i] = hl / 6.0;
            B[i] = (hl + hr) / 3.0;
            C[i] = hr / 6.0;
            D[i] = ((i > 0) ? lr[i - 1].y : 0.0) + ((i < N) ? lr[i].x : 0.0);
        }
        __syncthreads();
        int s = 1;
        for (; 2 * s - 1 < n; s <<= 1) {
            for (int i = 2 * s - 1 + 2 * s * threadIdx.x; i < n; i += 2 * s * blockDim.x) {
                const int l = i - s, r = i + s;
                const double alpha = -A[i] / B[l];
                double an = alpha * A[l];
                double bn = B[i] + alpha * C[l];
                double dn = D[i] + alpha * D[l];
                double cn = 0.0;
                if (r < n) {
                    const double gamma = -C[i] / B[r];
                    cn = gamma * C[r];
                    bn += gamma * A[r];
                    dn += gamma * D[r];
                }
                A[i] = an;
                B[i] = bn;
                C[i] = cn;
                D[i] = dn;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) D[s - 1] = D[s - 1] / B[s - 1];
        __syncthreads();
        for (s >>= 1; s >= 1; s >>= 1) {
            for (int i = s - 1 + 2 * s * threadIdx.x; i < n; i += 2 * s * blockDim.x) {
                double v = D[i];
                if (i - s >= 0) v -= A[i] * D[i - s];
                if (i + s < n) v -= C[i] * D[i + s];
                D[i] = v / B[i];
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) p.values[k0 + i] = D[i];
        __syncthreads();
    }
}

__global__ void single_project_setup_kernel(pwl_func F, int64_t N, pwl_func* funcs, int64_t* koff)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        funcs[0] = F;
        koff[0] = 0;
        koff[1] = N + 1;
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Gauss-Legendre nodes and weights on [-1, 1] for Q points: roots of the
// Legendre polynomial P_Q by Newton's method (P_Q and its derivative from
// Bonnet's recurrence), weights 2 / ((1 - x^2) P_Q'(x)^2).
void legendre_rule(int Q, double* xs, double* ws)
{
    for (int r = 0; r < (Q + 1) / 2; ++r) {
        double z = cos(M_PI * (r + 0.75) / (Q + 0.5));  // r-th largest root, initial guess
        double dP = 0.0;
        for (int it = 0; it < 64; ++it) {
            double Pm1 = 1.0, P = z;  // P_0, P_1
            for (int n = 2; n <= Q; ++n) {
                double Pn = ((2 * n - 1) * z * P - (n - 1) * Pm1) / n;
                Pm1 = P;
                P = Pn;
            }
            if (Q == 1) { P = z; Pm1 = 1.0; }
            dP = Q * (Pm1 - z * P) / (1.0 - z * z);
            double dz = P / dP;
            z -= dz;
            if (fabs(dz) <= 1e-17) break;
        }
        double Pm1 = 1.0, P = z;
        for (int n = 2; n <= Q; ++n) {
            double Pn = ((2 * n - 1) * z * P - (n - 1) * Pm1) / n;
            Pm1 = P;
            P = Pn;
        }
        if (Q == 1) { P = z; Pm1 = 1.0; }
        dP = Q * (Pm1 - z * P) / (1.0 - z * z);
        const double w = 2.0 / ((1.0 - z * z) * dP * dP);
        xs[Q - 1 - r] = z;
        ws[Q - 1 - r] = w;
        xs[r] = -z;
        ws[r] = w;
    }
    if (Q % 2 == 1) xs[Q / 2] = 0.0;
}

}  // namespace

const GaussLegendre& gauss_legendre_rule(int Q)
{
    static GaussLegendre rules[17];
    static std::once_flag once;
    std::call_once(once, [] {
        for (int q = 1; q <= 16; ++q) {
            rules[q].Q = q;
            legendre_rule(q, rules[q].x, rules[q].w);
            for (int i = 0; i < q; ++i) {
                rules[q].wl[i] = rules[q].w[i] * (1.0 - rules[q].x[i]) * 0.5;
                rules[q].wr[i] = rules[q].w[i] * (1.0 + rules[q].x[i]) * 0.5;
                rules[q].xf[i] = (float)rules[q].x[i];
            }
        }
    });
    return rules[Q];
}

size_t project_scratch_bytes(int64_t total_knots, int64_t total_intervals)
{
    return align256(sizeof(double2) * (size_t)total_intervals) +
           align256(sizeof(double) * 4 * (size_t)total_knots);
}

void project_carve_scratch(ProjectPlan& p, void* scratch)
{
    char* w = static_cast<char*>(scratch);
    p.lr = reinterpret_cast<double2*>(w);
    w += align256(sizeof(double2) * (size_t)p.total_intervals);
    p.cr = reinterpret_cast<double*>(w);
}

pwl_status project_launch(const ProjectPlan& p, const GaussLegendre& gl, cudaStream_t s)
{
    const DeviceInfo& di = device_info();
    if (p.form == PWL_INTERP) {
        const int grid = (int)std::min<int64_t>((p.total_knots + 255) / 256, (int64_t)di.sms * 16);
        if (p.precision == PWL_PREC_FP32)
            interp_values_kernel<float><<<grid, 256, 0, s>>>(p);
        else
            interp_values_kernel<double><<<grid, 256, 0, s>>>(p);
        PWL_CHECK_LAUNCH("interp_values_kernel");
        return PWL_OK;
    }
    const int grid = (int)std::min<int64_t>((p.total_intervals + 127) / 128, (int64_t)di.sms * 16);
    if (p.precision == PWL_PREC_FP32)
        hat_integrals_kernel<float><<<grid, 128, 0, s>>>(p, gl);
    else
        hat_integrals_kernel<double><<<grid, 128, 0, s>>>(p, gl);
    PWL_CHECK_LAUNCH("hat_integrals_kernel");
    if (p.solver == 1) {
        const int grid_t = (int)std::min<int64_t>((p.F + 63) / 64, (int64_t)di.sms * 16);
        gram_thomas_kernel<<<grid_t, 64, 0, s>>>(p);
        PWL_CHECK_LAUNCH("gram_thomas_kernel");
        return PWL_OK;
    }
    const size_t smem = sizeof(double) * 4 * (size_t)p.max_rows;
    const int use_smem = smem <= di.smem_optin ? 1 : 0;
    if (use_smem) {
        PWL_CUDA_TRY(cudaFuncSetAttribute(gram_solve_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    gram_solve_kernel<<<(int)std::min<int64_t>(p.F, 65535), kSolveThreads, use_smem ? smem : 0, s>>>(
        p, use_smem);
    PWL_CHECK_LAUNCH("gram_solve_kernel");
    return PWL_OK;
}

}  // namespace pwl

using namespace pwl;

namespace {
constexpr size_t kProjMeta = 256;
}

extern "C" {

size_t pwl_project_workspace_size(int64_t n_intervals)
{
    if (n_intervals < 1) return 0;
    return kProjMeta + project_scratch_bytes(n_intervals + 1, n_intervals);
}

pwl_status pwl_project(const pwl_func* f, const double* d_knots, int64_t n_intervals,
                       int32_t form, int32_t quad_points, int32_t precision, double* d_values,
                       void* d_workspace, size_t workspace_bytes, void* stream)
{
    clear_error();
    pwl_status st = validate_func(f);
    if (st != PWL_OK) return st;
    if (n_intervals < 1 || n_intervals > kMaxIntervals)
        return fail(PWL_EINVAL, "n_intervals must be in [1, %d]", kMaxIntervals);
    if (form != PWL_INTERP && form != PWL_PROJECT) return fail(PWL_EINVAL, "unknown form %d", form);
    if (quad_points == 0) quad_points = 8;
    if (quad_points < 1 || quad_points > 16)
        return fail(PWL_EINVAL, "quad_points must be in [1, 16] (got %d)", quad_points);
    if (precision != PWL_PREC_FP64 && precision != PWL_PREC_FP32)
        return fail(PWL_EINVAL, "unknown precision %d", precision);
    if (!d_knots || !d_values) return fail(PWL_EINVAL, "d_knots / d_values is NULL");
    const size_t need = pwl_project_workspace_size(n_intervals);
    if (!d_workspace || workspace_bytes < need)
        return fail(PWL_EINVAL, "workspace of %zu bytes needed (got %zu)", need, workspace_bytes);
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0)
        return fail(PWL_EINVAL, "workspace must be 256-byte aligned");
    char* w = static_cast<char*>(d_workspace);
    ProjectPlan p{};
    p.F = 1;
    p.precision = precision;
    p.form = form;
    p.max_rows = (int)(n_intervals + 1);
    p.total_knots = n_intervals + 1;
    p.total_intervals = n_intervals;
    p.funcs = reinterpret_cast<pwl_func*>(w);
    p.koff = reinterpret_cast<int64_t*>(w + 128);
    p.knots = d_knots;
    p.values = d_values;
    project_carve_scratch(p, w + kProjMeta);
    cudaStream_t s = as_stream(stream);
    single_project_setup_kernel<<<1, 1, 0, s>>>(*f, n_intervals, const_cast<pwl_func*>(p.funcs),
                                                const_cast<int64_t*>(p.koff));
    PWL_CHECK_LAUNCH("single_project_setup_kernel");
    return project_launch(p, gauss_legendre_rule(quad_points), s);
}

}  // extern "C"
