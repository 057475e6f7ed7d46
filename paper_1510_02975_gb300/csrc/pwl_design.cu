// pwl_design.cu -- knot placement for the nearly optimal partition T*
// (Section III-B): the local knot density |f''|^{2/5} (Eq. 16) on M uniform
// cells, its FP64 cumulative sum (the numerator of Eq. 18 by the midpoint
// rule) and the inversion F(x_i) = i/N (Eq. 17).
//
// Every kernel is batched over F functions described by device arrays
// (descriptors and CSR offsets of knots, cells and 2048-cell chunks); a
// single function is a batch of one.  Four launches:
//   density_chunks  d_k = |f''(t_k)|^{2/5} and one FP64 partial sum per chunk
//   chunk_scan      exclusive FP64 scan of the chunk sums, per function
//   cumulative      G_k = delta * (chunk base + in-chunk exclusive scan)
//   invert          one thread per knot: binary search of tau_i = i G_M / N
//                   in G, then the linear solve inside the cell
#include <math.h>

#include <algorithm>

#include "pwl_design.cuh"

namespace pwl {

namespace {

constexpr int kChunk = 2048;      // density cells per chunk
constexpr int kDesignThreads = 256;
constexpr int kPerThread = kChunk / kDesignThreads;

// index f with off[f] <= g < off[f+1] (off has F+1 non-decreasing entries)
__device__ __forceinline__ int find_segment(const int64_t* __restrict__ off, int F, int64_t g)
{
    int lo = 0, hi = F - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide exclusive scan of one double per thread (kDesignThreads
// threads).  Returns the exclusive prefix; *total receives the block sum.
__device__ __forceinline__ double block_exclusive_scan(double v, double* s_warp, double* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int W = kDesignThreads / 32;
    double incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        double t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    double excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) excl = 0.0;
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        double ws = (lane < W) ? s_warp[lane] : 0.0;
        double wi = ws;
        for (int o = 1; o < 32; o <<= 1) {
            double t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        double we = __shfl_up_sync(0xffffffffu, wi, 1);
        if (lane == 0) we = 0.0;
        if (lane < W) s_warp[lane] = we;
        if (lane == W - 1) s_warp[W] = wi;
    }
    __syncthreads();
    double r = s_warp[warp] + excl;
    *total = s_warp[W];
    __syncthreads();
    return r;
}

template <typename T>
__global__ void __launch_bounds__(kDesignThreads) density_chunks_kernel(DesignPlan p)
{
    __shared__ double s_red[kDesignThreads / 32];
    for (int64_t ch = blockIdx.x; ch < p.total_chunks; ch += gridDim.x) {
        const int f = find_segment(p.choff, p.F, ch);
        const pwl_func F = p.funcs[f];
        const int64_t M = p.moff[f + 1] - p.moff[f];
        const int64_t c0 = (ch - p.choff[f]) * kChunk;
        const double delta = (F.b - F.a) / (double)M;
        double* __restrict__ d = p.d + p.moff[f];
        double acc = 0.0;
        for (int r = 0; r < kPerThread; ++r) {
            const int64_t k = c0 + r * kDesignThreads + threadIdx.x;
            if (k < M) {
                // t_k = a + (k + 1/2) delta, rounded as written (no fused multiply-add)
                const double t = __dadd_rn(F.a, __dmul_rn((double)k + 0.5, delta));
                const T f2 = func_second_derivative<T>(F, (T)t);
                const double dk = (double)FMath<T>::pw(fabs(f2), T(0.4));
                d[k] = dk;
                acc += dk;
            }
        }
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < kDesignThreads / 32; ++w) s += s_red[w];
            p.csum[ch] = s;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kDesignThreads) chunk_scan_kernel(DesignPlan p)
{
    __shared__ double s_warp[kDesignThreads / 32 + 1];
    for (int f = blockIdx.x; f < p.F; f += gridDim.x) {
        const int64_t c0 = p.choff[f], c1 = p.choff[f + 1];
        double carry = 0.0;
        for (int64_t base = c0; base < c1; base += kDesignThreads) {
            const int64_t c = base + threadIdx.x;
            const double v = (c < c1) ? p.csum[c] : 0.0;
            double tot;
            const double ex = block_exclusive_scan(v, s_warp, &tot);
            if (c < c1) p.cbase[c] = carry + ex;
            carry += tot;
        }
        if (threadIdx.x == 0) p.stot[f] = carry;
    }
}

__global__ void __launch_bounds__(kDesignThreads) cumulative_kernel(DesignPlan p)
{
    __shared__ double s_d[kChunk];
    __shared__ double s_warp[kDesignThreads / 32 + 1];
    for (int64_t ch = blockIdx.x; ch < p.total_chunks; ch += gridDim.x) {
        const int f = find_segment(p.choff, p.F, ch);
        const int64_t M = p.moff[f + 1] - p.moff[f];
        const int64_t c0 = (ch - p.choff[f]) * kChunk;
        const int cnt = (int)min((int64_t)kChunk, M - c0);
        const double delta = (p.funcs[f].b - p.funcs[f].a) / (double)M;
        const double* __restrict__ d = p.d + p.moff[f];
        double* __restrict__ G = p.G + p.moff[f] + f;
        for (int i = threadIdx.x; i < kChunk; i += kDesignThreads) s_d[i] = (i < cnt) ? d[c0 + i] : 0.0;
        __syncthreads();
        double loc[kPerThread];
        double run = 0.0;
        for (int r = 0; r < kPerThread; ++r) {
            loc[r] = run;
            run += s_d[threadIdx.x * kPerThread + r];
        }
        double tot;
        const double tb = block_exclusive_scan(run, s_warp, &tot);
        const double base = p.cbase[ch] + tb;
        for (int r = 0; r < kPerThread; ++r) {
            const int i = threadIdx.x * kPerThread + r;
            if (i < cnt) G[c0 + i] = delta * (base + loc[r]);
        }
        if (c0 + cnt == M && threadIdx.x == 0) G[M] = delta * p.stot[f];
        __syncthreads();
    }
}

__global__ void invert_kernel(DesignPlan p)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < p.total_knots; g += stride) {
        const int f = find_segment(p.koff, p.F, g);
        const int64_t i = g - p.koff[f];
        const int64_t N = p.koff[f + 1] - p.koff[f] - 1;
        const double a = p.funcs[f].a, b = p.funcs[f].b;
        double x;
        if (i == 0) {
            x = a;
        } else if (i == N) {
            x = b;
        } else {
            const int64_t M = p.moff[f + 1] - p.moff[f];
            const double* __restrict__ G = p.G + p.moff[f] + f;
            const double* __restrict__ d = p.d + p.moff[f];
            const double GM = G[M];
            if (!(GM > 0.0)) {
                x = a + (double)i * (b - a) / (double)N;  // f linear on I: uniform partition
            } else {
                const double delta = (b - a) / (double)M;
                const double tau = (double)i * GM / (double)N;
                int64_t lo = 0, hi = M - 1;  // largest k with G_k <= tau
                while (lo < hi) {
                    const int64_t mid = lo + (hi - lo + 1) / 2;
                    if (G[mid] <= tau) lo = mid; else hi = mid - 1;
                }
                int64_t k = lo;
                while (k > 0 && !(d[k] > 0.0)) --k;
                x = __dadd_rn(a, __dmul_rn((double)k, delta));
                if (d[k] > 0.0) {
                    double step = (tau - G[k]) / d[k];
                    step = fmin(fmax(step, 0.0), delta);
                    x = __dadd_rn(x, step);
                }
            }
        }
        p.knots[g] = x;
    }
}

// Writes the descriptor and offsets of a one-function batch into the
// workspace (kernel parameters, so the call needs no host-to-device copy).
__global__ void single_setup_kernel(pwl_func F, int64_t N, int64_t M, pwl_func* funcs,
                                    int64_t* koff, int64_t* moff, int64_t* choff)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        funcs[0] = F;
        koff[0] = 0;
        koff[1] = N + 1;
        moff[0] = 0;
        moff[1] = M;
        choff[0] = 0;
        choff[1] = (M + kChunk - 1) / kChunk;
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

int64_t design_chunks(int64_t M) { return (M + kChunk - 1) / kChunk; }

size_t design_scratch_bytes(int64_t F, int64_t total_cells, int64_t total_chunks)
{
    return align256(sizeof(double) * (size_t)total_cells) +
           align256(sizeof(double) * (size_t)(total_cells + F)) +
           align256(sizeof(double) * (size_t)total_chunks) * 2 + align256(sizeof(double) * (size_t)F);
}

void design_carve_scratch(DesignPlan& p, void* scratch)
{
    char* w = static_cast<char*>(scratch);
    p.d = reinterpret_cast<double*>(w);
    w += align256(sizeof(double) * (size_t)p.total_cells);
    p.G = reinterpret_cast<double*>(w);
    w += align256(sizeof(double) * (size_t)(p.total_cells + p.F));
    p.csum = reinterpret_cast<double*>(w);
    w += align256(sizeof(double) * (size_t)p.total_chunks);
    p.cbase = reinterpret_cast<double*>(w);
    w += align256(sizeof(double) * (size_t)p.total_chunks);
    p.stot = reinterpret_cast<double*>(w);
}

pwl_status design_launch(const DesignPlan& p, cudaStream_t s)
{
    const DeviceInfo& di = device_info();
    const int grid_chunks = (int)std::min<int64_t>(p.total_chunks, (int64_t)di.sms * 8);
    if (p.precision == PWL_PREC_FP32)
        density_chunks_kernel<float><<<grid_chunks, kDesignThreads, 0, s>>>(p);
    else
        density_chunks_kernel<double><<<grid_chunks, kDesignThreads, 0, s>>>(p);
    PWL_CHECK_LAUNCH("density_chunks_kernel");
    chunk_scan_kernel<<<(int)std::min<int64_t>(p.F, 65535), kDesignThreads, 0, s>>>(p);
    PWL_CHECK_LAUNCH("chunk_scan_kernel");
    cumulative_kernel<<<grid_chunks, kDesignThreads, 0, s>>>(p);
    PWL_CHECK_LAUNCH("cumulative_kernel");
    const int grid_knots = (int)std::min<int64_t>((p.total_knots + 255) / 256, (int64_t)di.sms * 16);
    invert_kernel<<<grid_knots, 256, 0, s>>>(p);
    PWL_CHECK_LAUNCH("invert_kernel");
    return PWL_OK;
}

}  // namespace pwl

using namespace pwl;

namespace {
constexpr size_t kMetaBytes = 512;  // descriptor + three offset pairs
int64_t resolve_cells(int64_t n, int64_t m) { return m > 0 ? m : 64 * n; }
}  // namespace

extern "C" {

size_t pwl_design_workspace_size(int64_t n_intervals, int64_t m_cells)
{
    if (n_intervals < 1) return 0;
    const int64_t M = resolve_cells(n_intervals, m_cells);
    return kMetaBytes + design_scratch_bytes(1, M, design_chunks(M));
}

pwl_status pwl_design(const pwl_func* f, int64_t n_intervals, int64_t m_cells, int32_t precision,
                      double* d_knots, void* d_workspace, size_t workspace_bytes, void* stream)
{
    clear_error();
    pwl_status st = validate_func(f);
    if (st != PWL_OK) return st;
    if (n_intervals < 1 || n_intervals > kMaxIntervals)
        return fail(PWL_EINVAL, "n_intervals must be in [1, %d] (got %lld)", kMaxIntervals,
                    (long long)n_intervals);
    if (m_cells < 0 || m_cells > (int64_t)1 << 32)
        return fail(PWL_EINVAL, "m_cells must be in [0, 2^32] (got %lld)", (long long)m_cells);
    if (precision != PWL_PREC_FP64 && precision != PWL_PREC_FP32)
        return fail(PWL_EINVAL, "unknown precision %d", precision);
    if (!d_knots) return fail(PWL_EINVAL, "d_knots is NULL");
    const int64_t M = resolve_cells(n_intervals, m_cells);
    const size_t need = pwl_design_workspace_size(n_intervals, m_cells);
    if (!d_workspace || workspace_bytes < need)
        return fail(PWL_EINVAL, "workspace of %zu bytes needed (got %zu)", need, workspace_bytes);
    if (reinterpret_cast<uintptr_t>(d_workspace) % 256 != 0)
        return fail(PWL_EINVAL, "workspace must be 256-byte aligned");

    char* w = static_cast<char*>(d_workspace);
    DesignPlan p{};
    p.F = 1;
    p.funcs = reinterpret_cast<pwl_func*>(w);
    p.koff = reinterpret_cast<int64_t*>(w + 128);
    p.moff = reinterpret_cast<int64_t*>(w + 160);
    p.choff = reinterpret_cast<int64_t*>(w + 192);
    p.total_knots = n_intervals + 1;
    p.total_cells = M;
    p.total_chunks = design_chunks(M);
    p.precision = precision;
    p.knots = d_knots;
    design_carve_scratch(p, w + kMetaBytes);
    cudaStream_t s = as_stream(stream);
    single_setup_kernel<<<1, 1, 0, s>>>(*f, n_intervals, M, const_cast<pwl_func*>(p.funcs),
                                        const_cast<int64_t*>(p.koff), const_cast<int64_t*>(p.moff),
                                        const_cast<int64_t*>(p.choff));
    PWL_CHECK_LAUNCH("single_setup_kernel");
    return design_launch(p, s);
}

}  // extern "C"
