// pwl_table.cu -- device representation of a CPWL function: the inputs of
// Algorithm 1 (knots x_samples and values v_samples) rounded to their storage
// types, plus uniform cell indexes over [x_0, x_N] whose records make the
// search step of Algorithm 1 a single lookup (see pwl_common.cuh).
//
// Build (all single-CTA kernels, one host synchronisation in between):
//   table_round_kernel    FP64 -> FP32 knots, values -> dtype (-> FP32),
//                         slopes, reciprocal lengths, validation, shortest
//                         interval
//   table_index_b_kernel  backward index: cell of every knot, chain slots,
//                         16-byte knot records
//   table_index_f_kernel  forward index: 8-byte cell records, side records
// The host picks both cell counts between the first kernel and the others
// from the shortest interval and the shared-memory budgets.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "pwl_design.cuh"
#include "pwl_table.cuh"

namespace pwl {

namespace {

constexpr int kBuildThreads = 1024;

__device__ __forceinline__ int block_exclusive_scan_int(int v, int* s_warp, int* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int ws = (lane < W) ? s_warp[lane] : 0;
        int wi = ws;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < W) s_warp[lane] = wi - ws;
        if (lane == W - 1) s_warp[32] = wi;
    }
    __syncthreads();
    int r = s_warp[warp] + incl - v;
    *total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kBuildThreads) table_round_kernel(
    const double* __restrict__ knots, const double* __restrict__ values, int N, int dtype, float* xk,
    float* vk, void* vstore, float* slope, float* inv_h, TableHeader* hdr, int check_ends, float a, float b)
{
    __shared__ int s_status;
    __shared__ unsigned s_hmin;
    if (threadIdx.x == 0) {
        s_status = 0;
        s_hmin = 0x7f7fffffu;  // FLT_MAX
    }
    __syncthreads();
    int st = 0;
    for (int i = threadIdx.x; i <= N; i += blockDim.x) {
        const float xf = __double2float_rn(knots[i]);
        const float vf = __double2float_rn(values[i]);
        float vq = vf;
        if (dtype == PWL_BF16) {
            __nv_bfloat16 q = __float2bfloat16_rn(vf);
            static_cast<__nv_bfloat16*>(vstore)[i] = q;
            vq = __bfloat162float(q);
        } else if (dtype == PWL_FP16) {
            __half q = __float2half_rn(vf);
            static_cast<__half*>(vstore)[i] = q;
            vq = __half2float(q);
        } else {
            static_cast<float*>(vstore)[i] = vf;
        }
        if (!isfinite(xf) || !isfinite(vq)) st |= 2;
        xk[i] = xf;
        vk[i] = vq;
    }
    __syncthreads();
    float hmin = 3.402823466e38f;
    for (int i = 1 + threadIdx.x; i <= N; i += blockDim.x) {
        const double h = (double)xk[i] - (double)xk[i - 1];
        if (!(h > 0.0)) st |= 1;
        // one Newton-refined reciprocal instead of two FP64 divisions (this
        // single-CTA kernel runs on one SM's FP64 pipe); h <= 0, flagged
        // above, keeps the division's inf and NaN
        const double r = h > 0.0 ? recip_newton(h) : 1.0 / h;
        const double s = ((double)vk[i] - (double)vk[i - 1]) * r;
        const float fs = __double2float_rn(s);
        const float fr = __double2float_rn(r);
        if (!isfinite(fs) || !isfinite(fr)) st |= 4;
        slope[i] = fs;
        inv_h[i] = fr;
        hmin = fminf(hmin, (float)h);
    }
    if (threadIdx.x == 0) {
        // end conventions: s_0 := s_1, s_{N+1} := s_N (same for 1/h)
        const double h1 = (double)xk[1] - (double)xk[0];
        const double hN = (double)xk[N] - (double)xk[N - 1];
        slope[0] = __double2float_rn(((double)vk[1] - (double)vk[0]) / h1);
        inv_h[0] = __double2float_rn(1.0 / h1);
        slope[N + 1] = __double2float_rn(((double)vk[N] - (double)vk[N - 1]) / hN);
        inv_h[N + 1] = __double2float_rn(1.0 / hN);
    }
    // an update keeps the cell grids of the build, which span [a, b]: the
    // rounded end knots must not move (bit 3 otherwise)
    if (check_ends && threadIdx.x == 0 && !(xk[0] == a && xk[N] == b)) st |= 8;
    if (st) atomicOr(&s_status, st);
    if (hmin > 0.0f) atomicMin(&s_hmin, __float_as_uint(hmin));
    else atomicMin(&s_hmin, 0u);
    __syncthreads();
    if (threadIdx.x == 0) {
        TableHeader h{};
        h.status = s_status;
        h.hmin_bits = s_hmin;
        *hdr = h;
    }
}

// first index j in [0, n) with c[j] >= v (n if none)
__device__ __forceinline__ int lower_bound_int(const int* c, int n, int v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (c[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Cells of all knots, and the largest number of extra knots in one cell.
__device__ void knot_cells(int N, int K, float inv_w, float off, const float* __restrict__ xk, int* cj,
                           int* s_maxchain)
{
    for (int j = threadIdx.x; j <= N; j += blockDim.x) cj[j] = cell_of(xk[j], inv_w, off, K);
    __syncthreads();
    int my_max = 0;
    for (int j = 1 + threadIdx.x; j <= N; j += blockDim.x)
        if (cj[j] == cj[j - 1]) my_max = max(my_max, j - lower_bound_int(cj, N + 1, cj[j]));
    if (my_max) atomicMax(s_maxchain, my_max);
    __syncthreads();
}

__global__ void __launch_bounds__(kBuildThreads) table_index_b_kernel(
    int N, int K, float inv_w, float off, const float* __restrict__ xk, const float* __restrict__ vk,
    const float* __restrict__ slope, const float* __restrict__ inv_h, int* cj, int* cpos, float4* rec16,
    float4* rec_b, TableHeader* hdr)
{
    __shared__ int s_warp[33];
    __shared__ int s_maxchain;
    if (threadIdx.x == 0) s_maxchain = 0;
    __syncthreads();
    knot_cells(N, K, inv_w, off, xk, cj, &s_maxchain);
    int carry = 0;
    for (int base = 0; base <= N; base += blockDim.x) {
        const int j = base + threadIdx.x;
        const int flag = (j <= N && j > 0 && cj[j] == cj[j - 1]) ? 1 : 0;
        int tot;
        const int ex = block_exclusive_scan_int(flag, s_warp, &tot);
        if (j <= N) cpos[j] = carry + ex;
        carry += tot;
    }
    const int n_chain = carry;
    __syncthreads();
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        const int lb = lower_bound_int(cj, N + 1, c);
        int j;
        bool chained = false;
        const bool knot_cell = lb <= N && cj[lb] == c;
        if (knot_cell) {
            j = lb;
            chained = (j < N && cj[j + 1] == c);
        } else {
            // cell 0 holds knot 0 and cell K-1 knot N, so 0 <= j < N here; the
            // clamp keeps the reads in range after an update that moved x_0
            // (status bit 3, reported by pwl_table_check)
            j = max(lb - 1, 0);
        }
        const float w = chained ? make_link(K + cpos[j + 1]) : slope[j + 1];
        rec16[c] = make_float4(xk[j], vk[j], slope[j], w);
        // a knot-free cell's queries all lie in interval j + 1 (the cell
        // function is monotone): its record carries that interval's 1/h
        rec_b[c] = knot_cell ? make_float4(xk[j], __int_as_float(j), slope[j], w)
                             : make_float4(xk[j], __uint_as_float(kInsideFlag | (uint32_t)j), inv_h[j + 1], w);
    }
    for (int j = 1 + threadIdx.x; j <= N; j += blockDim.x) {
        if (cj[j] != cj[j - 1]) continue;
        const bool chained = (j < N && cj[j + 1] == cj[j]);
        const float w = chained ? make_link(K + cpos[j + 1]) : slope[j + 1];
        rec16[K + cpos[j]] = make_float4(xk[j], vk[j], slope[j], w);
        rec_b[K + cpos[j]] = make_float4(xk[j], __int_as_float(j), slope[j], w);
    }
    if (threadIdx.x == 0) {
        hdr->n_chain_b = n_chain;
        hdr->max_chain_b = s_maxchain;
    }
}

__global__ void __launch_bounds__(kBuildThreads) table_index_f_kernel(
    int N, int K, float inv_w, float off, float w, float a, const float* __restrict__ xk,
    const float* __restrict__ vk, const float* __restrict__ slope, int* cj, float2* recP, float2* recS,
    float2* recS8, TableHeader* hdr)
{
    __shared__ int s_maxchain;
    __shared__ int s_nchain;
    if (threadIdx.x == 0) {
        s_maxchain = 0;
        s_nchain = 0;
    }
    __syncthreads();
    knot_cells(N, K, inv_w, off, xk, cj, &s_maxchain);
    int my_chain = 0;
    for (int j = 1 + threadIdx.x; j <= N; j += blockDim.x) my_chain += (cj[j] == cj[j - 1]) ? 1 : 0;
    if (my_chain) atomicAdd(&s_nchain, my_chain);
    for (int c = threadIdx.x; c < K; c += blockDim.x) {
        const int lb = lower_bound_int(cj, N + 1, c);
        if (lb <= N && cj[lb] == c) {
            const bool chain = (lb < N && cj[lb + 1] == c);
            recP[c] = make_float2(make_knot_tag(lb, chain), xk[lb]);
        } else {
            // the line of interval j+1 through (x_j, v_j) with its FP32 slope,
            // valued at the anchor x_c (FP32: one FP64 division per cell would
            // dominate the build on this GPU's few FP64 units)
            const int j = max(lb - 1, 0);  // >= 0 unless an update moved x_0 (status bit 3)
            const float xc = __fmaf_rn(__int2float_rn(c), w, a);
            const float s = slope[j + 1];
            recP[c] = make_float2(__fmaf_rn(__fsub_rn(xc, xk[j]), s, vk[j]), s);
        }
    }
    for (int k = threadIdx.x; k <= N; k += blockDim.x) {
        recS[2 * k] = make_float2(vk[k], slope[k]);
        recS[2 * k + 1] = make_float2(vk[k], slope[k + 1]);
        recS8[k] = make_float2(vk[k], slope[k + 1]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        hdr->n_chain_f = s_nchain;
        hdr->max_chain_f = s_maxchain;
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

pwl_status launch_build(pwl_table t, const double* d_knots, const double* d_values, bool index_only,
                        cudaStream_t s)
{
    const int N = (int)t->N;
    if (!index_only) {
        table_round_kernel<<<1, kBuildThreads, 0, s>>>(d_knots, d_values, N, t->dtype, t->xk, t->vk, t->vstore,
                                                       t->slope, t->inv_h, t->hdr, 1, t->a, t->b);
        PWL_CHECK_LAUNCH("table_round_kernel");
    }
    table_index_b_kernel<<<1, kBuildThreads, 0, s>>>(N, (int)t->Kb, t->inv_w_b, t->off_b, t->xk, t->vk, t->slope,
                                                     t->inv_h, t->cj, t->cpos, t->rec16, t->rec_b, t->hdr);
    PWL_CHECK_LAUNCH("table_index_b_kernel");
    table_index_f_kernel<<<1, kBuildThreads, 0, s>>>(N, (int)t->K, t->inv_w, t->off, t->w, t->a, t->xk, t->vk,
                                                     t->slope, t->cj, t->recP, t->recS, t->recS8, t->hdr);
    PWL_CHECK_LAUNCH("table_index_f_kernel");
    return PWL_OK;
}

pwl_status status_error(const TableHeader& h)
{
    if (h.status & 1) return fail(PWL_EINVAL, "knots are not strictly increasing after rounding to FP32");
    if (h.status & 2) return fail(PWL_EINVAL, "a knot or value is not finite");
    if (h.status & 4) return fail(PWL_EINVAL, "a slope or reciprocal length overflows FP32");
    if (h.status & 8)
        return fail(PWL_EINVAL, "an update moved the end knots x_0 or x_N (after rounding to FP32); the table "
                                "keeps the cell grid of its build over [x_0, x_N]: build a new table instead");
    return PWL_OK;
}

}  // namespace

int64_t forward_cell_capacity(int64_t N, size_t budget)
{
    const size_t side = forward_side_bytes(N);
    const size_t fixed = forward_side_staged(N) ? side : 0;
    if (fixed + 8 * 64 > budget) return 64;
    return (int64_t)((budget - fixed) / sizeof(float2));
}

int64_t backward_cell_capacity(int64_t N)
{
    const size_t optin = device_info().smem_optin;
    const size_t fixed = 12 * (size_t)(N + 2) + 8 * 1024;  // reciprocal lengths, accumulators, chains
    if (fixed + 16 * 64 > optin) return (int64_t)((optin - 8 * 1024) / sizeof(float4));
    return (int64_t)((optin - fixed) / sizeof(float4));
}

void choose_cells(pwl_table t, float hmin, int64_t requested)
{
    const DeviceInfo& di = device_info();
    const int64_t N = t->N;
    // cells no wider than the shortest interval hold at most one knot
    const double need = ceil(((double)t->b - (double)t->a) / (double)hmin) + 1.0;
    // 8-byte index: worth its second, dependent gather on knot cells only
    // when it lets two CTAs share an SM while most cells (>= 3/4) are
    // knot-free and no cell holds two knots; otherwise the 16-byte index
    // serves the forward path too.  Two CTAs keep to kTwoCtaIndexBytes each:
    // beyond it the shared-memory carve-out of two CTAs leaves the L1 ~28 KB
    // for the streaming loads in flight (measured: ~5.55 TB/s at 102-113 KB
    // per CTA against ~6.5 TB/s at 86-96 KB, the same tables).
    constexpr size_t kTwoCtaIndexBytes = 96 * 1024;
    const size_t half = std::min<size_t>(di.smem_per_sm / 2 - 1024, kTwoCtaIndexBytes);
    const int64_t cap2 = forward_cell_capacity(N, half);
    const int64_t cap1 = forward_cell_capacity(N, di.smem_optin);
    const double want = std::max<double>(need, 8.0 * (double)(N + 1));
    int64_t K;
    if (requested > 0) {
        K = std::min<int64_t>(requested, cap1);
        t->layout = (K <= cap2 && K >= 4 * (N + 1)) ? 0 : 1;
    } else if ((double)cap2 >= std::max<double>(need, 4.0 * (double)(N + 1))) {
        K = (int64_t)std::min<double>(want, (double)cap2);
        t->layout = 0;
    } else {
        // one CTA per SM: the 8-byte index still wins while it stays chain-free
        // with >= 3 cells per knot inside kOneCtaIndexBytes (the carve-out then
        // leaves the L1 ~60 KB; at ~206 KB it drops to ~28 KB: Gaussian
        // N = 4096, 6.2 TB/s at 190 KB against 5.35 TB/s at 206 KB and
        // 5.95 TB/s on the 16-byte index)
        constexpr size_t kOneCtaIndexBytes = 190 * 1024;
        const size_t one = std::min<size_t>(di.smem_optin, kOneCtaIndexBytes);
        const int64_t cap1b = forward_cell_capacity(N, one);
        // the same budget with one side record per knot instead of two
        const size_t side8 = sizeof(float2) * (size_t)(N + 1);
        const int64_t cap1c = side8 + 8 * 1024 <= one ? (int64_t)((one - side8) / sizeof(float2)) : 0;
        const double min_cells = std::max<double>(need, 3.0 * (double)(N + 1));
        if ((double)cap1b >= min_cells) {
            K = (int64_t)std::min<double>(want, (double)cap1b);
            t->layout = 0;
        } else if ((double)cap1c >= min_cells) {
            // (the Lorentzian N = 4096 table: 20.1 K chain-free cells in 190 KB,
            // where two side records per knot left room for 15.5 K)
            K = (int64_t)std::min<double>(want, (double)cap1c);
            t->layout = 2;
        } else {
            K = (int64_t)std::min<double>(want, (double)cap1);
            t->layout = 1;
        }
    }
    t->K = std::max<int64_t>(K, 1);
    const int64_t capb = backward_cell_capacity(N);
    int64_t Kb = (requested > 0) ? std::min<int64_t>(requested, capb)
                                 : (int64_t)std::min<double>(std::max<double>(need, 2.0 * (double)(N + 1)),
                                                              (double)capb);
    t->Kb = std::max<int64_t>(std::min<int64_t>(Kb, (int64_t)kLinkMask - N - 2), 1);
    // cell functions c = trunc(fma(x, inv_w, off)), inv_w = K / (b - a);
    // 8-byte-index anchors x_c = fma(c, w, a), w = (b - a) / K
    t->inv_w = (float)t->K / (t->b - t->a);
    t->off = -t->a * t->inv_w;
    t->w = (t->b - t->a) / (float)t->K;
    t->inv_w_b = (float)t->Kb / (t->b - t->a);
    t->off_b = -t->a * t->inv_w_b;
}

}  // namespace pwl

using namespace pwl;

extern "C" {

pwl_status pwl_table_build(const double* d_knots, const double* d_values, int64_t n_intervals,
                           int32_t value_dtype, int64_t k_cells, pwl_table* out, void* stream)
{
    clear_error();
    if (!out) return fail(PWL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d_knots || !d_values) return fail(PWL_EINVAL, "d_knots / d_values is NULL");
    if (n_intervals < 1 || n_intervals > kMaxIntervals)
        return fail(PWL_EINVAL, "n_intervals must be in [1, %d] (got %lld)", kMaxIntervals,
                    (long long)n_intervals);
    if (value_dtype != PWL_FP32 && value_dtype != PWL_BF16 && value_dtype != PWL_FP16)
        return fail(PWL_EINVAL, "unknown value dtype %d", value_dtype);
    if (k_cells < 0) return fail(PWL_EINVAL, "k_cells must be >= 0");
    const int N = (int)n_intervals;
    cudaStream_t s = as_stream(stream);

    pwl_table_s* t = new (std::nothrow) pwl_table_s();
    if (!t) return fail(PWL_ENOMEM, "host allocation failed");
    memset(t, 0, sizeof(*t));
    cudaGetDevice(&t->device);
    t->N = N;
    t->dtype = value_dtype;
    const size_t n1 = (size_t)N + 1, n2 = (size_t)N + 2;
    const size_t o_xk = 256;
    const size_t o_vk = o_xk + align256(4 * n1);
    const size_t o_sl = o_vk + align256(4 * n1);
    const size_t o_ih = o_sl + align256(4 * n2);
    const size_t o_vs = o_ih + align256(4 * n2);
    const size_t o_cj = o_vs + align256(4 * n1);
    const size_t o_cp = o_cj + align256(4 * n1);
    const size_t total = o_cp + align256(4 * n1);
    cudaError_t e = dev_malloc(&t->buf_base, total);
    if (e != cudaSuccess) {
        delete t;
        return cuda_fail(e, "cudaMalloc(table)");
    }
    char* base = static_cast<char*>(t->buf_base);
    t->hdr = reinterpret_cast<TableHeader*>(base);
    t->xk = reinterpret_cast<float*>(base + o_xk);
    t->vk = reinterpret_cast<float*>(base + o_vk);
    t->slope = reinterpret_cast<float*>(base + o_sl);
    t->inv_h = reinterpret_cast<float*>(base + o_ih);
    t->vstore = base + o_vs;
    t->cj = reinterpret_cast<int*>(base + o_cj);
    t->cpos = reinterpret_cast<int*>(base + o_cp);

    auto bail = [&](pwl_status st) {
        pwl_table_destroy(t);
        return st;
    };

    table_round_kernel<<<1, kBuildThreads, 0, s>>>(d_knots, d_values, N, value_dtype, t->xk, t->vk,
                                                   t->vstore, t->slope, t->inv_h, t->hdr, 0, 0.0f, 0.0f);
    if ((e = cudaGetLastError()) != cudaSuccess) return bail(cuda_fail(e, "table_round_kernel"));
    TableHeader h{};
    float ab[2];
    if ((e = cudaMemcpyAsync(&h, t->hdr, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&ab[0], t->xk, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&ab[1], t->xk + N, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return bail(cuda_fail(e, "table build (rounding pass)"));
    pwl_status st = status_error(h);
    if (st != PWL_OK) return bail(st);
    float hmin;
    memcpy(&hmin, &h.hmin_bits, 4);
    t->a = ab[0];
    t->b = ab[1];
    choose_cells(t, hmin, k_cells);
    const size_t bytes_b = align256(sizeof(float4) * ((size_t)t->Kb + n1));
    const size_t bytes_p = align256(sizeof(float2) * (size_t)t->K);
    const size_t bytes_s = align256(sizeof(float2) * 2 * n1);
    const size_t bytes_s8 = align256(sizeof(float2) * n1);
    if ((e = dev_malloc(&t->buf_rec, 2 * bytes_b + bytes_p + bytes_s + bytes_s8)) != cudaSuccess)
        return bail(cuda_fail(e, "cudaMalloc(records)"));
    char* r = static_cast<char*>(t->buf_rec);
    t->rec_b = reinterpret_cast<float4*>(r);
    t->rec16 = reinterpret_cast<float4*>(r + bytes_b);
    t->recP = reinterpret_cast<float2*>(r + 2 * bytes_b);
    t->recS = reinterpret_cast<float2*>(r + 2 * bytes_b + bytes_p);
    t->recS8 = reinterpret_cast<float2*>(r + 2 * bytes_b + bytes_p + bytes_s);
    if ((st = launch_build(t, d_knots, d_values, true, s)) != PWL_OK) return bail(st);
    if ((e = cudaMemcpyAsync(&h, t->hdr, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return bail(cuda_fail(e, "table build (index pass)"));
    t->n_chain_b = h.n_chain_b;
    t->n_chain_f = h.n_chain_f;
    // chains in the 16-byte index (cells holding several knots) cost more than
    // the 8-byte index's single-CTA occupancy when the latter has none
    if (t->layout == 1 && k_cells == 0 && t->n_chain_b > 0 && t->n_chain_f == 0) t->layout = 0;
    // shared-memory room for the chains of this build and of later updates
    // that move a few knots (further chain records are read from global memory)
    t->chain_reserve_b = std::min<int64_t>((int64_t)n1, t->n_chain_b + 64);
    *out = t;
    return PWL_OK;
}

pwl_status pwl_table_update(pwl_table t, const double* d_knots, const double* d_values, void* stream)
{
    clear_error();
    if (!t) return fail(PWL_EINVAL, "table is NULL");
    if (!d_knots || !d_values) return fail(PWL_EINVAL, "d_knots / d_values is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return fail(PWL_EINVAL, "table lives on device %d, current device is %d", t->device, dev);
    const pwl_status st = launch_build(t, d_knots, d_values, false, as_stream(stream));
    if (st != PWL_OK) return st;
    return refresh_texture(t, as_stream(stream));
}

pwl_status pwl_table_check(pwl_table t, void* stream)
{
    clear_error();
    if (!t) return fail(PWL_EINVAL, "table is NULL");
    TableHeader h{};
    cudaStream_t s = as_stream(stream);
    PWL_CUDA_TRY(cudaMemcpyAsync(&h, t->hdr, sizeof(h), cudaMemcpyDeviceToHost, s));
    PWL_CUDA_TRY(cudaStreamSynchronize(s));
    return status_error(h);
}

pwl_status pwl_table_destroy(pwl_table t)
{
    if (!t) return PWL_OK;
    if (t->tex) cudaDestroyTextureObject(t->tex);
    if (t->tex_array) cudaFreeArray(t->tex_array);
    if (t->buf_rec) cudaFree(t->buf_rec);
    if (t->buf_base) cudaFree(t->buf_base);
    delete t;
    return PWL_OK;
}

pwl_status pwl_table_get_info(pwl_table t, pwl_table_info* info)
{
    clear_error();
    if (!t || !info) return fail(PWL_EINVAL, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->n_intervals = t->N;
    info->k_cells = t->K;
    info->n_chain = t->n_chain_f;
    info->value_dtype = t->dtype;
    info->a = t->a;
    info->b = t->b;
    info->d_knots = t->xk;
    info->d_values = t->vstore;
    info->eval_smem_bytes =
        t->layout == 0 ? eval8_smem_bytes(t) : (t->layout == 2 ? eval8c_smem_bytes(t) : eval16_smem_bytes(t));
    info->layout = t->layout;
    info->backward_smem_bytes = backward_smem_bytes(t);
    return PWL_OK;
}

}  // extern "C"
