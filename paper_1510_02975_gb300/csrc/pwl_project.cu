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

template <typename T, bool SAMPLED>
__global__ void interp_values_kernel(ProjectPlan p)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < p.total_knots; g += stride) {
        const int f = find_knot_owner(p.koff, p.F, g);
        const pwl_func F = p.funcs[f];
        if ((F.kind == PWL_F_SAMPLED) != SAMPLED) continue;  // the other launch's
        p.values[g] = (double)func_value_k<SAMPLED, T>(F, (T)p.knots[g]);
    }
}

// (L_j, R_j) = (int_{I_j} f phi_{j-1}, int_{I_j} f phi_j) for every interval.
// At the node t_q = mid + half x_q the hats are phi_{j-1} = (1 - x_q)/2 and
// phi_j = (1 + x_q)/2, so L_j = half sum_q wl_q f(t_q) and
// R_j = half sum_q wr_q f(t_q) with the host-side weights wl, wr: no
// division per node.  FP64 mode: t_q and the sums in FP64.  FP32 mode: t_q
// and f(t_q) in FP32 (the argument of an FP32 f is rounded to FP32 anyway),
// the sums in FP64.
// sum_q wl_q f(t_q) and sum_q wr_q f(t_q) over one interval (the half-length
// factor applied by the caller); the sampled path is a template flag,
// chosen once per interval
template <typename T, bool SAMPLED>
__device__ __forceinline__ void hat_sums(const pwl_func& F, const GaussLegendre& gl, double mid, double half,
                                         double& L, double& R)
{
    if constexpr (sizeof(T) == 4) {
        // sums of w f(t) as float-float pairs: each product exact (the
        // weight split hi + lo, the rounding error of hi f recovered by an
        // FMA), each addition compensated; FP64 once per interval
        const float midf = (float)mid, halff = (float)half;
        float Lh = 0.0f, Ll = 0.0f, Rh = 0.0f, Rl = 0.0f;
        auto acc = [](float& h, float& l, float wh, float wlo, float fv) {
            const float p = __fmul_rn(wh, fv);
            const float pe = __fmaf_rn(wh, fv, -p) + __fmul_rn(wlo, fv);  // hi f - p exactly, plus lo f
            const float s = __fadd_rn(h, p);
            const float bp = __fsub_rn(s, h);
            const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(p, bp));
            h = s;
            l = __fadd_rn(l, __fadd_rn(e, pe));
        };
        for (int q = 0; q < gl.Q; ++q) {
            const float fv = func_value_k<SAMPLED, float>(F, __fmaf_rn(halff, gl.xf[q], midf));
            acc(Lh, Ll, gl.wlh[q], gl.wll[q], fv);
            acc(Rh, Rl, gl.wrh[q], gl.wrl[q], fv);
        }
        L = (double)Lh + (double)Ll;
        R = (double)Rh + (double)Rl;
    } else {
        L = 0.0;
        R = 0.0;
        for (int q = 0; q < gl.Q; ++q) {
            const double fv = func_value_k<SAMPLED, double>(F, __fma_rn(half, gl.x[q], mid));
            L = __fma_rn(gl.wl[q], fv, L);
            R = __fma_rn(gl.wr[q], fv, R);
        }
    }
}

template <typename T, bool SAMPLED>
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
        if ((F.kind == PWL_F_SAMPLED) != SAMPLED) continue;  // the other launch's
        double L, R;
        hat_sums<T, SAMPLED>(F, gl, mid, half, L, R);
        p.lr[g] = make_double2(half * L, half * R);
    }
}

// Gram system of a batch of functions, one warp per function, by a
// partitioned Thomas algorithm (the SPIKE decomposition):
//  1. lane p owns rows r0_p .. r1_p - 1 (m >= 2 rows; P <= 32 segments) and
//     runs the Thomas elimination of its block with three right-hand sides:
//     the load vector (solution y), the coupling a_{r0} e_0 to the unknown
//     before the block (spike v) and the coupling c_{r1-1} e_{m-1} to the
//     unknown after it (spike w), so that on the block x = y - v L_{p-1}
//     - w F_{p+1}, with F_p, L_p the block's first and last unknowns;
//  2. the 2P boundary unknowns follow from the first and last rows of every
//     block: with L_{p-1} = alpha_{p-1} + beta_{p-1} F_p eliminated forward,
//     F_p = gamma_p + delta_p F_{p+1}, then F and L backward from F_P = 0
//     (a 2P-step recurrence in lane order, FP64; the spikes are below 1 in
//     magnitude on this diagonally dominant matrix, so every pivot
//     1 + v0_p beta_{p-1} stays near 1);
//  3. every lane reconstructs its rows.
// The rows are assembled on the fly (M_{i,i-1} = h_i/6, M_ii = (h_i +
// h_{i+1})/3, M_{i,i+1} = h_{i+1}/6, b_i = R_i + L_{i+1}).  About 20 FP64
// operations per row, one division; no barrier beyond the warp.

__global__ void __launch_bounds__(64) gram_spike_kernel(ProjectPlan p, const int* __restrict__ order)
{
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    constexpr double kSixth = 1.0 / 6.0, kThird = 1.0 / 3.0;
    for (int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); o < p.F; o += warps) {
        const int f = order ? order[o] : o;
        const int64_t k0 = p.koff[f];
        const int n = (int)(p.koff[f + 1] - k0);
        const int N = n - 1;
        const double* __restrict__ x = p.knots + k0;
        const double2* __restrict__ lr = p.lr + (k0 - f);
        double* __restrict__ sc = p.cr + 4 * k0;  // per row: c', then y, v, w
        const int P = min(32, max(1, n / 2));
        double y0 = 0.0, v0 = 0.0, w0 = 0.0, yL = 0.0, vL = 0.0, wL = 0.0;
        const int r0 = (int)((int64_t)lane * n / P), r1 = (int)((int64_t)(lane + 1) * n / P);
        if (lane < P) {
            // forward elimination of the block, three right-hand sides
            double cprev = 0.0, yprev = 0.0, vprev = 0.0, wlast = 0.0;
            // the interval left of row i carries over from the previous row
            double xi = x[r0];
            double hl = r0 > 0 ? xi - x[r0 - 1] : 0.0;
#pragma unroll 4
            for (int i = r0; i < r1; ++i) {
                const double xn = i < N ? x[i + 1] : xi;
                const double hr = xn - xi;
                const double rhs = (i > 0 ? lr[i - 1].y : 0.0) + (i < N ? lr[i].x : 0.0);
                const double lower = i > r0 ? hl * kSixth : 0.0;  // coupling inside the block
                const double upper = hr * kSixth;
                const double r = recip_newton((hl + hr) * kThird - lower * cprev);
                const double yv = (rhs - lower * yprev) * r;
                const double vv = ((i == r0 ? hl * kSixth : 0.0) - lower * vprev) * r;
                cprev = i + 1 < r1 ? upper * r : 0.0;
                if (i + 1 == r1) wlast = upper * r;  // w'_{m-1}: the coupling to the next block
                sc[4 * i] = cprev;
                sc[4 * i + 1] = yv;
                sc[4 * i + 2] = vv;
                yprev = yv;
                vprev = vv;
                hl = hr;
                xi = xn;
            }
            // back substitution: y_j, v_j, w_j (w' is zero above the last row)
            double yn = 0.0, vn = 0.0, wn = 0.0;
#pragma unroll 4
            for (int i = r1 - 1; i >= r0; --i) {
                const double c = sc[4 * i];
                const double yv = sc[4 * i + 1] - c * yn;
                const double vv = sc[4 * i + 2] - c * vn;
                const double wv = (i == r1 - 1 ? wlast : 0.0) - c * wn;
                sc[4 * i + 1] = yv;
                sc[4 * i + 2] = vv;
                sc[4 * i + 3] = wv;
                yn = yv;
                vn = vv;
                wn = wv;
                if (i == r1 - 1) {
                    yL = yv;
                    vL = vv;
                    wL = wv;
                }
            }
            y0 = yn;
            v0 = vn;
            w0 = wn;
        }
        // boundary unknowns, forward over the blocks in lane order.  Every lane
        // runs the same recurrence on shuffled (uniform) inputs; lane q keeps
        // block q's coefficients.  Carried: L_{q-1} = alpha + beta F_q.
        double alpha = 0.0, beta = 0.0;
        double gq_own = 0.0, dq_own = 0.0, aq_own = 0.0, bq_own = 0.0;
        for (int q = 0; q < P; ++q) {
            const double y0q = __shfl_sync(0xffffffffu, y0, q), v0q = __shfl_sync(0xffffffffu, v0, q);
            const double w0q = __shfl_sync(0xffffffffu, w0, q), yLq = __shfl_sync(0xffffffffu, yL, q);
            const double vLq = __shfl_sync(0xffffffffu, vL, q), wLq = __shfl_sync(0xffffffffu, wL, q);
            // F_q = y0 - v0 L_{q-1} - w0 F_{q+1}  ->  F_q = g + d F_{q+1}
            const double piv = 1.0 / (1.0 + v0q * beta);
            const double g = (y0q - v0q * alpha) * piv;
            const double d = -w0q * piv;
            // L_q = yL - vL L_{q-1} - wL F_{q+1}  ->  L_q = an + bn F_{q+1}
            const double an = yLq - vLq * (alpha + beta * g);
            const double bn = -(vLq * beta * d + wLq);
            if (lane == q) {
                gq_own = g;
                dq_own = d;
                aq_own = an;
                bq_own = bn;
            }
            alpha = an;
            beta = bn;
        }
        // backward from F_P = 0: F_q = g_q + d_q F_{q+1}, L_q = a_q + b_q F_{q+1}
        double Fnext = 0.0, Fq = 0.0, Lq = 0.0;
        for (int q = P - 1; q >= 0; --q) {
            const double gq = __shfl_sync(0xffffffffu, gq_own, q), dq = __shfl_sync(0xffffffffu, dq_own, q);
            const double aq = __shfl_sync(0xffffffffu, aq_own, q), bq = __shfl_sync(0xffffffffu, bq_own, q);
            if (lane == q) {
                Fq = Fnext;  // F_{q+1}, the unknown after this lane's block
                Lq = aq + bq * Fnext;
            }
            Fnext = gq + dq * Fnext;
        }
        // L_{p-1} from the previous lane (0 before the first block)
        double Lprev = __shfl_up_sync(0xffffffffu, Lq, 1);
        if (lane == 0) Lprev = 0.0;
        if (lane < P) {
            double* __restrict__ v = p.values + k0;
#pragma unroll 4
            for (int i = r0; i < r1; ++i) v[i] = sc[4 * i + 1] - sc[4 * i + 2] * Lprev - sc[4 * i + 3] * Fq;
        }
    }
}

// Gram system of the hat basis and its solution by cyclic reduction.  Rows
// 0..n-1 (n = N+1).  Forward: for strides s = 1, 2, 4, ... while 2s-1 < n,
// every row i = 2s-1 (mod 2s) eliminates its couplings to rows i-s and i+s
// (coefficients a: to i-s, c: to i+s).  One row (s_top - 1) is then
// uncoupled; back substitution fills rows s-1 (mod 2s) for s = s_top/2..1.
// One CTA solves one function, so the solve runs on a single SM's FP64
// pipe: the pivots' reciprocals come from recip_newton (five FP64
// operations) and the entries from products with 1/6 and 1/3, not from
// FP64 divisions (the bench's design graph 0.495 -> 0.455 ms).
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
            A[i] = hl * (1.0 / 6.0);
            B[i] = (hl + hr) * (1.0 / 3.0);
            C[i] = hr * (1.0 / 6.0);
            D[i] = ((i > 0) ? lr[i - 1].y : 0.0) + ((i < N) ? lr[i].x : 0.0);
        }
        __syncthreads();
        int s = 1;
        for (; 2 * s - 1 < n; s <<= 1) {
            for (int i = 2 * s - 1 + 2 * s * threadIdx.x; i < n; i += 2 * s * blockDim.x) {
                const int l = i - s, r = i + s;
                const double alpha = -A[i] * recip_newton(B[l]);
                double an = alpha * A[l];
                double bn = B[i] + alpha * C[l];
                double dn = D[i] + alpha * D[l];
                double cn = 0.0;
                if (r < n) {
                    const double gamma = -C[i] * recip_newton(B[r]);
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
        if (threadIdx.x == 0) D[s - 1] = D[s - 1] * recip_newton(B[s - 1]);
        __syncthreads();
        for (s >>= 1; s >= 1; s >>= 1) {
            for (int i = s - 1 + 2 * s * threadIdx.x; i < n; i += 2 * s * blockDim.x) {
                double v = D[i];
                if (i - s >= 0) v -= A[i] * D[i - s];
                if (i + s < n) v -= C[i] * D[i + s];
                D[i] = v * recip_newton(B[i]);
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
                rules[q].wlh[i] = (float)rules[q].wl[i];
                rules[q].wll[i] = (float)(rules[q].wl[i] - (double)rules[q].wlh[i]);
                rules[q].wrh[i] = (float)rules[q].wr[i];
                rules[q].wrl[i] = (float)(rules[q].wr[i] - (double)rules[q].wrh[i]);
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
        const int kinds = plan_kinds(p.kinds);
        if (kinds & kKindsAnalytic) {
            if (p.precision == PWL_PREC_FP32)
                interp_values_kernel<float, false><<<grid, 256, 0, s>>>(p);
            else
                interp_values_kernel<double, false><<<grid, 256, 0, s>>>(p);
            PWL_CHECK_LAUNCH("interp_values_kernel");
        }
        if (kinds & kKindsSampled) {
            if (p.precision == PWL_PREC_FP32)
                interp_values_kernel<float, true><<<grid, 256, 0, s>>>(p);
            else
                interp_values_kernel<double, true><<<grid, 256, 0, s>>>(p);
            PWL_CHECK_LAUNCH("interp_values_kernel");
        }
        return PWL_OK;
    }
    const int grid = (int)std::min<int64_t>((p.total_intervals + 127) / 128, (int64_t)di.sms * 16);
    const int kinds = plan_kinds(p.kinds);
    if (kinds & kKindsAnalytic) {
        if (p.precision == PWL_PREC_FP32)
            hat_integrals_kernel<float, false><<<grid, 128, 0, s>>>(p, gl);
        else
            hat_integrals_kernel<double, false><<<grid, 128, 0, s>>>(p, gl);
        PWL_CHECK_LAUNCH("hat_integrals_kernel");
    }
    if (kinds & kKindsSampled) {
        if (p.precision == PWL_PREC_FP32)
            hat_integrals_kernel<float, true><<<grid, 128, 0, s>>>(p, gl);
        else
            hat_integrals_kernel<double, true><<<grid, 128, 0, s>>>(p, gl);
        PWL_CHECK_LAUNCH("hat_integrals_kernel");
    }
    if (p.solver == 1) {
        // two warps (functions) per CTA, so that a few hundred functions
        // still spread over every SM
        const int grid_w = (int)std::min<int64_t>((p.F + 1) / 2, (int64_t)di.sms * 32);
        gram_spike_kernel<<<grid_w, 64, 0, s>>>(p, p.order);
        PWL_CHECK_LAUNCH("gram_spike_kernel");
        return PWL_OK;
    }
    const size_t smem = sizeof(double) * 4 * (size_t)p.max_rows;
    const int use_smem = smem <= di.smem_optin ? 1 : 0;
    if (use_smem) {
        PWL_CUDA_TRY(raise_smem_limit(gram_solve_kernel, smem));
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
    p.kinds = kinds_of(f, 1);
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
