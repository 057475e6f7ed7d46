// pwl_eval.cu -- CPWL evaluation (Algorithm 1) over a query stream.
//
// Main path (pwl_eval): a persistent grid; every CTA stages the table's cell
// records in shared memory, then streams 16-byte vectors of queries with
// several loads in flight per thread.  Per query: clamp to [x_0, x_N], one
// fma + truncation for the cell (step 1 of Algorithm 1 reduced to a lookup),
// one 16-byte shared-memory load of the record, a select between the two
// slopes, and v_j + (x - x_j) * s (steps 2-3 fused into one FMA).  Cells
// that hold several knots chain to further records (rare by construction).
//
// Comparison paths (pwl_eval_variant):
//   mode 0  the paper's Algorithm 1: binary search over the FP32 knots in
//           shared memory (Section IV), delta, (1 - delta) v_{i-1} + delta v_i
//   mode 1  the same interval lookup as the main path, then the texture
//           unit's linear filter at i - 1 + delta + 1/2 (Section IV-B).
#include <math.h>

#include <algorithm>

#include "pwl_table.cuh"

namespace pwl {

namespace {

constexpr int kUnroll = 4;

struct EvalArgs {
    const float4* rec;
    const TableHeader* hdr;
    int K;
    int n_smem;     // records staged in shared memory (at launch: the room reserved)
    int max_chain;  // chain hops (set from the device header by the kernel)
    float a, b, inv_w, off;
    int64_t head;  // scalar queries before the first 16-byte boundary of x
    int64_t nvec;  // 16-byte vectors after the head
};

template <bool CHAINS>
__device__ __forceinline__ float lerp_one(float x, const float4* __restrict__ srec, const EvalArgs& p)
{
    const float xc = clamp_nan(x, p.a, p.b);
    const int c = cell_of(xc, p.inv_w, p.off, p.K);
    float4 r = srec[c];
    if (CHAINS) {
        for (int g = 0; g < p.max_chain && xc > r.x && is_link(r.w); ++g) {
            const int j = link_index(r.w);
            r = (j < p.n_smem) ? srec[j] : __ldg(p.rec + j);
        }
    }
    // x == x_j takes the left slope: v_j + 0 * s_j is exactly v_j
    const float s = (xc <= r.x) ? r.z : r.w;
    return __fmaf_rn(xc - r.x, s, r.y);
}

// 16-byte vectors of each I/O type
template <typename IO>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int n = 4;
    using T = float4;
    template <bool C>
    static __device__ __forceinline__ T apply(T v, const float4* s, const EvalArgs& p)
    {
        v.x = lerp_one<C>(v.x, s, p);
        v.y = lerp_one<C>(v.y, s, p);
        v.z = lerp_one<C>(v.z, s, p);
        v.w = lerp_one<C>(v.w, s, p);
        return v;
    }
    static __device__ __forceinline__ float to_f(float x) { return x; }
    static __device__ __forceinline__ float from_f(float x) { return x; }
};
template <>
struct Vec<__nv_bfloat16> {
    static constexpr int n = 8;
    using T = uint4;
    template <bool C>
    static __device__ __forceinline__ T apply(T v, const float4* s, const EvalArgs& p)
    {
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 f = __bfloat1622float2(h[k]);
            f.x = lerp_one<C>(f.x, s, p);
            f.y = lerp_one<C>(f.y, s, p);
            h[k] = __float22bfloat162_rn(f);
        }
        return v;
    }
    static __device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
    static __device__ __forceinline__ __nv_bfloat16 from_f(float x) { return __float2bfloat16_rn(x); }
};
template <>
struct Vec<__half> {
    static constexpr int n = 8;
    using T = uint4;
    template <bool C>
    static __device__ __forceinline__ T apply(T v, const float4* s, const EvalArgs& p)
    {
        __half2* h = reinterpret_cast<__half2*>(&v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 f = __half22float2(h[k]);
            f.x = lerp_one<C>(f.x, s, p);
            f.y = lerp_one<C>(f.y, s, p);
            h[k] = __float22half2_rn(f);
        }
        return v;
    }
    static __device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
    static __device__ __forceinline__ __half from_f(float x) { return __float2half_rn(x); }
};

// streaming (evict-first) 16-byte global accesses
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }
__device__ __forceinline__ uint4 ld_stream(const uint4* p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(float4* p, float4 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(uint4* p, uint4 v) { __stcs(p, v); }

template <typename IO, bool CHAINS>
__device__ __forceinline__ void eval_body(const EvalArgs& p, const float4* __restrict__ srec, const IO* x,
                                          IO* y, int64_t m)
{
    using V = Vec<IO>;
    using T = typename V::T;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const T* xv = reinterpret_cast<const T*>(x + p.head);
    T* yv = reinterpret_cast<T*>(y + p.head);
    int64_t i = tid;
    for (; i + (kUnroll - 1) * nthr < p.nvec; i += kUnroll * nthr) {
        T v[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) v[u] = ld_stream(xv + i + u * nthr);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) v[u] = V::template apply<CHAINS>(v[u], srec, p);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) st_stream(yv + i + u * nthr, v[u]);
    }
    for (; i < p.nvec; i += nthr) st_stream(yv + i, V::template apply<CHAINS>(ld_stream(xv + i), srec, p));
    for (int64_t j = tid; j < p.head; j += nthr) y[j] = V::from_f(lerp_one<CHAINS>(V::to_f(x[j]), srec, p));
    for (int64_t j = p.head + p.nvec * V::n + tid; j < m; j += nthr)
        y[j] = V::from_f(lerp_one<CHAINS>(V::to_f(x[j]), srec, p));
}

// MINB = 2 asks for <= 32 registers so that two 1024-thread CTAs fit an SM
// (used when two copies of the records fit its shared memory).
template <typename IO, int MINB>
__global__ void __launch_bounds__(1024, MINB) eval_kernel(const EvalArgs args, const IO* x, IO* y, int64_t m)
{
    extern __shared__ float4 srec[];
    EvalArgs p = args;
    const int n_chain = p.hdr->n_chain;
    p.max_chain = p.hdr->max_chain;
    p.n_smem = min(p.K + n_chain, p.n_smem);  // the rest of the chain area stays in global memory
    for (int i = threadIdx.x; i < p.n_smem; i += blockDim.x) srec[i] = __ldg(p.rec + i);
    __syncthreads();
    if (n_chain == 0)
        eval_body<IO, false>(p, srec, x, y, m);
    else
        eval_body<IO, true>(p, srec, x, y, m);
}

// ---- mode 0: Algorithm 1 with a binary search over the knots --------------
__global__ void __launch_bounds__(1024) eval_search_kernel(const float* __restrict__ xk_g,
                                                           const float* __restrict__ vk_g, int N,
                                                           const float* x, float* y, int64_t m)
{
    extern __shared__ float2 s_kv[];  // (x_j, v_j)
    for (int j = threadIdx.x; j <= N; j += blockDim.x) s_kv[j] = make_float2(xk_g[j], vk_g[j]);
    __syncthreads();
    const float a = s_kv[0].x, b = s_kv[N].x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += nthr) {
        const float xc = clamp_nan(__ldcs(x + q), a, b);
        // upper bound: first knot > x, over [0, N+1), clamped to [1, N]
        int lo = 0, hi = N + 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_kv[mid].x > xc) hi = mid; else lo = mid + 1;
        }
        const int i = min(max(lo, 1), N);
        const float2 l = s_kv[i - 1], r = s_kv[i];
        const float delta = (xc - l.x) / (r.x - l.x);
        __stcs(y + q, (1.0f - delta) * l.y + delta * r.y);
    }
}

// ---- mode 1: interval lookup, then the texture unit's linear filter -------
__global__ void __launch_bounds__(1024) eval_tex_kernel(const EvalArgs args, const float* __restrict__ inv_h_g,
                                                        int N, cudaTextureObject_t tex, const float* x,
                                                        float* y, int64_t m)
{
    extern __shared__ float4 s_dyn[];
    float4* srec = s_dyn;                                          // backward-form records
    float* s_ih = reinterpret_cast<float*>(s_dyn + args.n_smem);   // N+2 reciprocal lengths
    EvalArgs p = args;
    p.max_chain = p.hdr->max_chain;
    p.n_smem = min(p.K + p.hdr->n_chain, p.n_smem);
    for (int i = threadIdx.x; i < p.n_smem; i += blockDim.x) srec[i] = __ldg(p.rec + i);
    for (int i = threadIdx.x; i < N + 2; i += blockDim.x) s_ih[i] = inv_h_g[i];
    __syncthreads();
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += nthr) {
        const float xc = clamp_nan(__ldcs(x + q), p.a, p.b);
        const int c = cell_of(xc, p.inv_w, p.off, p.K);
        float4 r = (c < p.n_smem) ? srec[c] : __ldg(p.rec + c);
        for (int g = 0; g < p.max_chain && xc >= r.x && is_link(r.w); ++g) {
            const int j = link_index(r.w);
            r = (j < p.n_smem) ? srec[j] : __ldg(p.rec + j);
        }
        const int j = __float_as_int(r.y);
        float u;  // texel coordinate i - 1 + delta + 1/2
        if (xc < r.x) {
            u = (float)j + 0.5f - (r.x - xc) * s_ih[j];
        } else if (j < N) {
            u = (float)j + 0.5f + (xc - r.x) * s_ih[j + 1];
        } else {
            u = (float)N + 0.5f;
        }
        float yv = tex1D<float>(tex, u);
        if (xc != xc) yv = xc;
        __stcs(y + q, yv);
    }
}

pwl_status check_common(pwl_table t, const void* x, const void* y, int64_t m)
{
    if (!t) return fail(PWL_EINVAL, "table is NULL");
    if (m < 0) return fail(PWL_EINVAL, "m must be >= 0");
    if (m > 0 && (!x || !y)) return fail(PWL_EINVAL, "x / y is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device)
        return fail(PWL_EINVAL, "table lives on device %d, current device is %d", t->device, dev);
    return PWL_OK;
}

EvalArgs make_args(pwl_table t, const float4* rec, int64_t n_smem)
{
    EvalArgs p{};
    p.rec = rec;
    p.hdr = t->hdr;
    p.K = (int)t->K;
    p.n_smem = (int)n_smem;
    p.max_chain = 0;
    p.a = t->a;
    p.b = t->b;
    p.inv_w = t->inv_w;
    p.off = t->off;
    return p;
}

template <typename IO>
pwl_status launch_eval(pwl_table t, const IO* x, IO* y, int64_t m, cudaStream_t s)
{
    const int64_t n_smem = eval_smem_records(t);
    if (n_smem < t->K) return fail(PWL_ENOTSUP, "cell index of %lld records does not fit one CTA", (long long)t->K);
    EvalArgs p = make_args(t, t->rec_f, n_smem);
    const uintptr_t ax = reinterpret_cast<uintptr_t>(x), ay = reinterpret_cast<uintptr_t>(y);
    if ((ax % 16) == (ay % 16) && (ax % sizeof(IO)) == 0) {
        const int64_t head = std::min<int64_t>(m, (int64_t)(((16 - ax % 16) % 16) / sizeof(IO)));
        p.head = head;
        p.nvec = (m - head) / Vec<IO>::n;
    } else {
        p.head = 0;
        p.nvec = 0;
    }
    const size_t smem = sizeof(float4) * (size_t)n_smem;
    const DeviceInfo& di = device_info();
    const bool two = di.smem_per_sm >= 2 * (smem + 1024);
    auto kern = two ? eval_kernel<IO, 2> : eval_kernel<IO, 1>;
    int max_grid = 0;
    PWL_CUDA_TRY(occupancy_grid(kern, 1024, smem, &max_grid));
    // no more CTAs than there are unrolled vector groups (small launches
    // should not stage the table in hundreds of idle CTAs)
    const int64_t units = p.nvec + (m - p.nvec * Vec<IO>::n);
    const int64_t per_cta = (int64_t)1024 * kUnroll;
    const int grid = (int)std::min<int64_t>(max_grid, std::max<int64_t>(1, (units + per_cta - 1) / per_cta));
    kern<<<grid, 1024, smem, s>>>(p, x, y, m);
    PWL_CHECK_LAUNCH("eval_kernel");
    return PWL_OK;
}

pwl_status ensure_texture(pwl_table t)
{
    if (t->tex) return PWL_OK;
    int maxw = 0;
    cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture1DLinearWidth, t->device);
    int maxa = 0;
    cudaDeviceGetAttribute(&maxa, cudaDevAttrMaxTexture1DWidth, t->device);
    if (t->N + 1 > maxa)
        return fail(PWL_ENOTSUP, "texture path supports at most %d knots", maxa);
    const bool half_texels = (t->dtype == PWL_FP16);
    cudaChannelFormatDesc cd = half_texels ? cudaCreateChannelDescHalf() : cudaCreateChannelDesc<float>();
    PWL_CUDA_TRY(cudaMallocArray(&t->tex_array, &cd, (size_t)t->N + 1, 0));
    const void* src = half_texels ? t->vstore : (const void*)t->vk;
    const size_t esz = half_texels ? 2 : 4;
    PWL_CUDA_TRY(cudaMemcpy2DToArray(t->tex_array, 0, 0, src, esz * (t->N + 1), esz * (t->N + 1), 1,
                                     cudaMemcpyDeviceToDevice));
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = t->tex_array;
    cudaTextureDesc td{};
    td.addressMode[0] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModeLinear;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    PWL_CUDA_TRY(cudaCreateTextureObject(&t->tex, &rd, &td, nullptr));
    return PWL_OK;
}

}  // namespace

}  // namespace pwl

using namespace pwl;

extern "C" {

pwl_status pwl_eval(pwl_table t, const void* d_x, void* d_y, int64_t m, int32_t io_dtype, void* stream)
{
    clear_error();
    pwl_status st = check_common(t, d_x, d_y, m);
    if (st != PWL_OK) return st;
    if (m == 0) return PWL_OK;
    cudaStream_t s = as_stream(stream);
    switch (io_dtype) {
    case PWL_FP32:
        return launch_eval<float>(t, static_cast<const float*>(d_x), static_cast<float*>(d_y), m, s);
    case PWL_BF16:
        return launch_eval<__nv_bfloat16>(t, static_cast<const __nv_bfloat16*>(d_x),
                                          static_cast<__nv_bfloat16*>(d_y), m, s);
    case PWL_FP16:
        return launch_eval<__half>(t, static_cast<const __half*>(d_x), static_cast<__half*>(d_y), m, s);
    }
    return fail(PWL_EINVAL, "unknown io dtype %d", io_dtype);
}

pwl_status pwl_eval_variant(pwl_table t, int32_t mode, const float* d_x, float* d_y, int64_t m,
                            void* stream)
{
    clear_error();
    pwl_status st = check_common(t, d_x, d_y, m);
    if (st != PWL_OK) return st;
    if (mode != 0 && mode != 1) return fail(PWL_EINVAL, "unknown mode %d", mode);
    if (m == 0) return PWL_OK;
    cudaStream_t s = as_stream(stream);
    const DeviceInfo& di = device_info();
    if (mode == 0) {
        const size_t smem = sizeof(float2) * (size_t)(t->N + 1);
        if (smem > di.smem_optin)
            return fail(PWL_ENOTSUP, "binary-search path stages N+1 <= %zu knots", di.smem_optin / 8);
        int grid = 0;
        PWL_CUDA_TRY(occupancy_grid(eval_search_kernel, 1024, smem, &grid));
        eval_search_kernel<<<grid, 1024, smem, s>>>(t->xk, t->vk, (int)t->N, d_x, d_y, m);
        PWL_CHECK_LAUNCH("eval_search_kernel");
        return PWL_OK;
    }
    st = ensure_texture(t);
    if (st != PWL_OK) return st;
    const size_t fixed = sizeof(float) * (size_t)(t->N + 2);
    if (fixed + 1024 > di.smem_optin) return fail(PWL_ENOTSUP, "table too large for the texture path");
    const int64_t n_smem = std::min<int64_t>(t->K + t->chain_reserve, (int64_t)((di.smem_optin - fixed) / 16));
    EvalArgs p = make_args(t, t->rec_b, n_smem);
    const size_t smem = 16 * (size_t)n_smem + fixed;
    int grid = 0;
    PWL_CUDA_TRY(occupancy_grid(eval_tex_kernel, 1024, smem, &grid));
    eval_tex_kernel<<<grid, 1024, smem, s>>>(p, t->inv_h, (int)t->N, t->tex, d_x, d_y, m);
    PWL_CHECK_LAUNCH("eval_tex_kernel");
    return PWL_OK;
}

}  // extern "C"
