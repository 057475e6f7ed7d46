// pwl_stream.cuh -- the streaming shape shared by every per-query kernel:
// a persistent grid walks the query stream in 16-byte vectors with several
// loads in flight per thread (loads at the L2 only, evict-first stores), with a scalar
// head before the first 16-byte boundary and a scalar tail; and the
// register-generated query stream of the compute-ceiling runs.
//
// A per-query kernel supplies a functor float -> float (the lookup and lerp
// of Algorithm 1, or a direct evaluation of f) and calls stream_body or
// synth_sum with it.
#pragma once

#include <algorithm>

#include "pwl_common.cuh"

namespace pwl {

// 16-byte vectors of each I/O type
template <typename IO>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int n = 4;
    using T = float4;
    template <class L>
    static __device__ __forceinline__ T apply(T v, const L& f)
    {
        v.x = f(v.x);
        v.y = f(v.y);
        v.z = f(v.z);
        v.w = f(v.w);
        return v;
    }
    static __device__ __forceinline__ float to_f(float x) { return x; }
    static __device__ __forceinline__ float from_f(float x) { return x; }
};
template <>
struct Vec<__nv_bfloat16> {
    static constexpr int n = 8;
    using T = uint4;
    template <class L>
    static __device__ __forceinline__ T apply(T v, const L& f)
    {
        __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 g = __bfloat1622float2(h[k]);
            g.x = f(g.x);
            g.y = f(g.y);
            h[k] = __float22bfloat162_rn(g);
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
    template <class L>
    static __device__ __forceinline__ T apply(T v, const L& f)
    {
        __half2* h = reinterpret_cast<__half2*>(&v);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 g = __half22float2(h[k]);
            g.x = f(g.x);
            g.y = f(g.y);
            h[k] = __float22half2_rn(g);
        }
        return v;
    }
    static __device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
    static __device__ __forceinline__ __half from_f(float x) { return __float2half_rn(x); }
};

// 16-byte global accesses of the stream: loads cached at the L2 only
// (ld.global.cg; 1% faster than evict-first loads), evict-first stores
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ uint4 ld_stream(const uint4* p) { return __ldcg(p); }
__device__ __forceinline__ void st_stream(float4* p, float4 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(uint4* p, uint4 v) { __stcs(p, v); }

// y[q] = f(x[q]) for q < m over the whole grid: `head` scalar queries up to
// the first 16-byte boundary of x (and of y: the launcher only takes the
// vector path when both share their alignment), `nvec` 16-byte vectors with
// U loads in flight per thread, then the scalar tail.
template <typename IO, int U, class L>
__device__ __forceinline__ void stream_body(int64_t head, int64_t nvec, const L& f, const IO* x, IO* y, int64_t m)
{
    using V = Vec<IO>;
    using T = typename V::T;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const T* xv = reinterpret_cast<const T*>(x + head);
    T* yv = reinterpret_cast<T*>(y + head);
    int64_t i = tid;
    for (; i + (U - 1) * nthr < nvec; i += U * nthr) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = ld_stream(xv + i + u * nthr);
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = V::apply(v[u], f);
#pragma unroll
        for (int u = 0; u < U; ++u) st_stream(yv + i + u * nthr, v[u]);
    }
    for (; i < nvec; i += nthr) st_stream(yv + i, V::apply(ld_stream(xv + i), f));
    for (int64_t j = tid; j < head; j += nthr) y[j] = V::from_f(f(V::to_f(x[j])));
    for (int64_t j = head + nvec * V::n + tid; j < m; j += nthr) y[j] = V::from_f(f(V::to_f(x[j])));
}

// Host side: the scalar head and the vector count of a stream of m elements
// (no vectors when x and y do not share their 16-byte alignment).
template <typename IO>
inline void stream_split(const void* x, const void* y, int64_t m, int64_t* head, int64_t* nvec)
{
    const uintptr_t ax = reinterpret_cast<uintptr_t>(x), ay = reinterpret_cast<uintptr_t>(y);
    if ((ax % 16) == (ay % 16) && (ax % sizeof(IO)) == 0) {
        *head = std::min<int64_t>(m, (int64_t)(((16 - ax % 16) % 16) / sizeof(IO)));
        *nvec = (m - *head) / Vec<IO>::n;
    } else {
        *head = 0;
        *nvec = 0;
    }
}

// Host side: CTAs of a streaming launch of `units` vectors and scalars with
// `threads` threads per CTA: no more than there are unrolled vector groups,
// but one per SM while each gets a few vectors per warp, and at most the
// persistent grid.
inline int stream_grid(int max_grid, int64_t units, int threads, int unroll)
{
    const int64_t per_cta = (int64_t)threads * unroll;
    const int64_t spread = std::min<int64_t>(device_info().sms, (units + 255) / 256);
    return (int)std::min<int64_t>(max_grid,
                                  std::max<int64_t>(1, std::max<int64_t>(spread, (units + per_cta - 1) / per_cta)));
}

// ---- the register-generated query stream (compute-ceiling runs) -----------
// u_q = top 24 bits of lowbias32(q + seed) / 2^24 (the 32-bit integer hash
// "lowbias32" of the hash-prospector project: xor-shift 16, multiply
// 0x7feb352d, xor-shift 15, multiply 0x846ca68b, xor-shift 16), and
// x_q = u_q (b - a) + a in FP32 (two roundings).
__device__ __forceinline__ uint32_t lowbias32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// This thread's FP32 sum of f over its share of the m generated queries.
template <class L>
__device__ __forceinline__ float synth_sum(const L& f, uint32_t seed, float a, float w, int64_t m)
{
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    float acc = 0.0f;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += nthr) {
        const float u = (float)(lowbias32((uint32_t)q + seed) >> 8) * 0x1p-24f;
        acc += f(__fadd_rn(__fmul_rn(u, w), a));
    }
    return acc;
}

// Adds the CTA's sum of every thread's acc to *sum (FP64).  s_red: at least
// 32 floats of shared memory that no thread reads any more (a barrier comes
// first).
__device__ __forceinline__ void cta_sum_to(float acc, float* s_red, double* sum)
{
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += (double)s_red[k];
        atomicAdd(sum, t);
    }
}

}  // namespace pwl
