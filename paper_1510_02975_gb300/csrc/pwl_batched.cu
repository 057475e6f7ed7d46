// pwl_batched.cu -- many independent functions with uneven knot and query
// counts: design, projection, index build and evaluation of a whole batch,
// each a fixed sequence of launches over all functions, so that the four
// phases can be captured in one CUDA graph and replayed.
//
//   design      density / chunk scan / cumulative / inversion over the chunks
//               of every function at once (the kernels of pwl_design.cu)
//   projection  hat integrals of every interval, then one CTA per function
//               for the Gram solve (pwl_project.cu)
//   index       one CTA per function: FP32 knots and values, slopes and the
//               8-byte cell index of the single-table path (pwl_common.cuh),
//               with a cell count per function that lets two CTAs share an SM
//   evaluation  one persistent launch.  The concatenated query stream is cut
//               into one contiguous range per CTA of about equal cost; a CTA
//               walks the functions of its range, staging a function's index
//               in shared memory when its share of that function's queries
//               pays for the copy, else reading the index through L1/L2.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "pwl_async.cuh"
#include "pwl_design.cuh"
#include "pwl_table.cuh"

namespace pwl {

namespace {

constexpr int kIndexThreads = 1024;
constexpr int kMaxBatchIntervals = 65535;

// Per-function data of the evaluation index (device).
struct BatchFunc {
    int64_t koff;  // first knot in the concatenated knot arrays (N+1 per function)
    int64_t soff;  // first slope (N+2 per function)
    int64_t poff;  // first cell record (K per function)
    int N, K;
    float a, b, inv_w, off, w;
    int n_chain, max_chain, status;
};

struct WorkItem {
    int f;
    int staged;      // 1: stage the index in shared memory
    int64_t q0, q1;  // query range (indices into x and y)
};

__device__ __forceinline__ int lower_bound_int(const int* c, int n, int v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (c[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// One CTA per function: FP32 knots and values, slopes, the cell of every
// knot, the K cell records and the 2 (N+1) side records.
__global__ void __launch_bounds__(kIndexThreads) batch_index_kernel(
    int F, const double* __restrict__ knots, const double* __restrict__ values, BatchFunc* bf, float* xk_all,
    float* vk_all, float* slope_all, int* cj_all, float2* recP, float2* recS)
{
    __shared__ int s_status, s_nchain, s_maxchain;
    for (int f = blockIdx.x; f < F; f += gridDim.x) {
        BatchFunc d = bf[f];
        const int N = d.N, K = d.K;
        float* x = xk_all + d.koff;
        float* v = vk_all + d.koff;
        float* s = slope_all + d.soff;
        int* cj = cj_all + d.koff;
        if (threadIdx.x == 0) {
            s_status = 0;
            s_nchain = 0;
            s_maxchain = 0;
        }
        __syncthreads();
        for (int i = threadIdx.x; i <= N; i += blockDim.x) {
            x[i] = __double2float_rn(knots[d.koff + i]);
            v[i] = __double2float_rn(values[d.koff + i]);
            if (!isfinite(x[i]) || !isfinite(v[i])) atomicOr(&s_status, 2);
        }
        __syncthreads();
        for (int i = 1 + threadIdx.x; i <= N; i += blockDim.x) {
            const float h = __fsub_rn(x[i], x[i - 1]);
            if (!(h > 0.0f)) atomicOr(&s_status, 1);
            s[i] = __fdiv_rn(__fsub_rn(v[i], v[i - 1]), h);
        }
        // every thread derives the same cell geometry from x_0 and x_N
        d.a = x[0];
        d.b = x[N];
        d.inv_w = __fdiv_rn((float)K, __fsub_rn(d.b, d.a));
        d.off = -d.a * d.inv_w;
        d.w = __fdiv_rn(__fsub_rn(d.b, d.a), (float)K);
        __syncthreads();
        if (threadIdx.x == 0) {
            s[0] = s[1];
            s[N + 1] = s[N];
        }
        for (int j = threadIdx.x; j <= N; j += blockDim.x) cj[j] = cell_of(x[j], d.inv_w, d.off, K);
        __syncthreads();
        int my_chain = 0, my_max = 0;
        for (int j = 1 + threadIdx.x; j <= N; j += blockDim.x) {
            if (cj[j] == cj[j - 1]) {
                ++my_chain;
                my_max = max(my_max, j - lower_bound_int(cj, N + 1, cj[j]));
            }
        }
        if (my_chain) atomicAdd(&s_nchain, my_chain);
        if (my_max) atomicMax(&s_maxchain, my_max);
        float2* P = recP + d.poff;
        float2* S = recS + 2 * d.koff;
        for (int c = threadIdx.x; c < K; c += blockDim.x) {
            const int lb = lower_bound_int(cj, N + 1, c);
            if (lb <= N && cj[lb] == c) {
                const bool chain = (lb < N && cj[lb + 1] == c);
                P[c] = make_float2(make_knot_tag(lb, chain), x[lb]);
            } else {
                // no knot in the cell: it lies inside interval lb, (x_{lb-1}, x_lb)
                const int j = lb - 1;
                const float xc = __fmaf_rn(__int2float_rn(c), d.w, d.a);
                P[c] = make_float2(__fmaf_rn(__fsub_rn(xc, x[j]), s[j + 1], v[j]), s[j + 1]);
            }
        }
        for (int k = threadIdx.x; k <= N; k += blockDim.x) {
            S[2 * k] = make_float2(v[k], s[k]);
            S[2 * k + 1] = make_float2(v[k], s[k + 1]);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            d.n_chain = s_nchain;
            d.max_chain = s_maxchain;
            d.status = s_status;
            bf[f] = d;
        }
        __syncthreads();
    }
}

// What the evaluation of one function needs per query.
struct Lookup {
    float a, b, inv_w, off, w;
    int K, N, max_chain;
};

// v(x) through the 8-byte index of one function; the arithmetic of the
// single-table forward path.  STAGED: P and S point to shared memory.
template <bool CHAINS, bool STAGED>
__device__ __forceinline__ float batch_lerp(float x, const Lookup& d, const float2* P, const float2* S,
                                            const float* __restrict__ xk)
{
    const float xc = clamp_nan(x, d.a, d.b);
    const int c = cell_of(xc, d.inv_w, d.off, d.K);
    const float2 r = STAGED ? P[c] : __ldg(P + c);
    const uint32_t bits = __float_as_uint(r.x);
    float anchor = __fmaf_rn(__int2float_rn(c), d.w, d.a);
    float2 q = r;
    if ((bits & 0xFFC00000u) == kLinkTag) {
        int k = (int)(bits & kKnotTagMask);
        float xkk = r.y;
        if (CHAINS && (bits & kKnotTagChain)) {
            for (int g = 0; g < d.max_chain && k < d.N; ++g) {
                const float xn = __ldg(xk + k + 1);
                if (!(xc >= xn)) break;
                ++k;
                xkk = xn;
            }
        }
        const int si = 2 * k + (xc >= xkk ? 1 : 0);
        q = STAGED ? S[si] : __ldg(S + si);
        anchor = xkk;
    }
    return __fmaf_rn(xc - anchor, q.y, q.x);
}

// Queries q0 .. q1-1 of one function (q1 - q0 < 2^31).
template <int U, bool CHAINS, bool STAGED>
__device__ __forceinline__ void batch_range(const Lookup& d, const float2* P, const float2* S, const float* xk,
                                            const float* __restrict__ x, float* __restrict__ y, int64_t q0,
                                            int64_t q1)
{
    // 16-byte vectors between the first and the last 16-byte boundary of the
    // range, scalar head and tail (fewer than 4 queries each).  The head and
    // tail loads go out first and complete while the vectors stream.  The
    // vectors are read at the L2 only (ld.global.cg): the staged index leaves
    // the L1 little room, and no other CTA reads the same lines.
    const int64_t v0 = min(q1, (q0 + 3) & ~(int64_t)3);
    const int64_t v1 = max(v0, q1 & ~(int64_t)3);
    const int nt = blockDim.x;
    const bool has_h = threadIdx.x < (int)(v0 - q0), has_t = threadIdx.x < (int)(q1 - v1);
    const float xh = has_h ? x[q0 + threadIdx.x] : 0.0f;
    const float xt = has_t ? x[v1 + threadIdx.x] : 0.0f;
    const float4* xv = reinterpret_cast<const float4*>(x + v0);
    float4* yv = reinterpret_cast<float4*>(y + v0);
    const int nv = (int)((v1 - v0) / 4);
    int i = threadIdx.x;
    for (; i + (U - 1) * nt < nv; i += U * nt) {
        float4 a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) a[u] = __ldcg(xv + i + u * nt);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            a[u].x = batch_lerp<CHAINS, STAGED>(a[u].x, d, P, S, xk);
            a[u].y = batch_lerp<CHAINS, STAGED>(a[u].y, d, P, S, xk);
            a[u].z = batch_lerp<CHAINS, STAGED>(a[u].z, d, P, S, xk);
            a[u].w = batch_lerp<CHAINS, STAGED>(a[u].w, d, P, S, xk);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) __stcs(yv + i + u * nt, a[u]);
    }
    for (; i < nv; i += nt) {
        float4 a = __ldcg(xv + i);
        a.x = batch_lerp<CHAINS, STAGED>(a.x, d, P, S, xk);
        a.y = batch_lerp<CHAINS, STAGED>(a.y, d, P, S, xk);
        a.z = batch_lerp<CHAINS, STAGED>(a.z, d, P, S, xk);
        a.w = batch_lerp<CHAINS, STAGED>(a.w, d, P, S, xk);
        __stcs(yv + i, a);
    }
    if (has_h) y[q0 + threadIdx.x] = batch_lerp<CHAINS, STAGED>(xh, d, P, S, xk);
    if (has_t) y[v1 + threadIdx.x] = batch_lerp<CHAINS, STAGED>(xt, d, P, S, xk);
}

// Queries q0 .. q1-1 of one function, the 16-byte vectors streamed through a
// per-thread ring of D slots in shared memory: thread t's k-th vector lands
// in slot ring[(k mod D) * blockDim + t] by cp.async, D vectors ahead of its
// use, so every thread keeps D - 1 to D loads in flight while it computes,
// whatever its register budget.  A slot is refilled only after its values
// have been consumed by the lerp (whose record loads depend on them).
template <int D, bool CHAINS, bool STAGED>
__device__ __forceinline__ void batch_range_ring(const Lookup& d, const float2* P, const float2* S,
                                                 const float* xk, const float* __restrict__ x,
                                                 float* __restrict__ y, int64_t q0, int64_t q1, float4* ring)
{
    static_assert((D & (D - 1)) == 0, "D is a power of two");
    const int64_t v0 = min(q1, (q0 + 3) & ~(int64_t)3);
    const int64_t v1 = max(v0, q1 & ~(int64_t)3);
    const int nt = blockDim.x, t = threadIdx.x;
    for (int j = t; j < (int)(v0 - q0); j += nt) y[q0 + j] = batch_lerp<CHAINS, STAGED>(x[q0 + j], d, P, S, xk);
    const float4* xv = reinterpret_cast<const float4*>(x + v0);
    float4* yv = reinterpret_cast<float4*>(y + v0);
    const int nv = (int)((v1 - v0) / 4);
    const int mine = nv > t ? (nv - 1 - t) / nt + 1 : 0;  // vectors t, t + nt, ... of this thread
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (k < mine) cp_async16(ring + k * nt + t, xv + t + (int64_t)k * nt);
        cp_async_commit();
    }
    for (int k = 0; k < mine; ++k) {
        cp_async_wait<D - 1>();  // the group of vector k has landed
        float4* slot = ring + (k & (D - 1)) * nt + t;
        float4 a = *slot;
        a.x = batch_lerp<CHAINS, STAGED>(a.x, d, P, S, xk);
        a.y = batch_lerp<CHAINS, STAGED>(a.y, d, P, S, xk);
        a.z = batch_lerp<CHAINS, STAGED>(a.z, d, P, S, xk);
        a.w = batch_lerp<CHAINS, STAGED>(a.w, d, P, S, xk);
        if (k + D < mine) cp_async16(slot, xv + t + (int64_t)(k + D) * nt);
        cp_async_commit();
        __stcs(yv + t + (int64_t)k * nt, a);
    }
    cp_async_wait<0>();
    for (int j = t; j < (int)(q1 - v1); j += nt) y[v1 + j] = batch_lerp<CHAINS, STAGED>(x[v1 + j], d, P, S, xk);
}

struct EvalParams {
    const WorkItem* items;
    const int* range;        // range r holds items range[r] .. range[r+1]-1
    int n_ranges;            // CTA b starts on range b, then takes gridDim + *counter++ (dynamic shapes)
    int* counter;            // zeroed before every launch
    const BatchFunc* bf;
    const float* xk_all;
    const float2* recP;
    const float2* recS;
    int buf_stride;          // float2 records per shared-memory buffer (asynchronous staging)
    int* status;             // device word: bit 2 set if a wait for a staging copy timed out
    uint64_t wait_ns;        // limit of one wait for a staging copy (asynchronous staging)
    int withheld;            // failure injection: arrivals a staging barrier expects but never gets (0 or 1)
};

__device__ __forceinline__ Lookup lookup_of(const BatchFunc& g)
{
    return Lookup{g.a, g.b, g.inv_w, g.off, g.w, g.K, g.N, g.max_chain};
}

// Streams one piece: U vectors in flight per thread from registers (D == 0)
// or a D-slot cp.async ring in shared memory.
template <int U, int D, bool STAGED>
__device__ __forceinline__ void run_piece(const EvalParams& p, const BatchFunc& g, const WorkItem& w,
                                          const float2* buf, const float* x, float* y, float4* ring)
{
    const Lookup d = lookup_of(g);
    const float2* P = STAGED ? buf : p.recP + g.poff;
    const float2* S = STAGED ? buf + g.K : p.recS + 2 * g.koff;
    const float* xk = p.xk_all + g.koff;
    if constexpr (D > 0) {
        if (g.n_chain)
            batch_range_ring<D, true, STAGED>(d, P, S, xk, x, y, w.q0, w.q1, ring);
        else
            batch_range_ring<D, false, STAGED>(d, P, S, xk, x, y, w.q0, w.q1, ring);
    } else {
        if (g.n_chain)
            batch_range<U, true, STAGED>(d, P, S, xk, x, y, w.q0, w.q1);
        else
            batch_range<U, false, STAGED>(d, P, S, xk, x, y, w.q0, w.q1);
    }
}

template <int U>
__device__ __forceinline__ void run_direct(const EvalParams& p, const BatchFunc& g, const WorkItem& w,
                                           const float* x, float* y)
{
    run_piece<U, 0, false>(p, g, w, nullptr, x, y, nullptr);
}

template <int U>
__device__ __forceinline__ void run_staged(const EvalParams& p, const BatchFunc& g, const WorkItem& w,
                                           const float2* buf, const float* x, float* y)
{
    run_piece<U, 0, true>(p, g, w, buf, x, y, nullptr);
}

// n float2 records from global memory into shared memory by the whole CTA,
// as cp.async copies that use no registers: every thread issues all of its
// copies (~5 for an average index) before one wait, so staging a function's
// index costs about one load latency instead of one per THREADS records.
// The copies are 16 bytes (two records) and skip the L1 (cp.async.cg): every
// function's cell records start 16-byte aligned and both arrays hold an even
// number of records (K is even).  The caller commits, waits and synchronises.
template <int THREADS>
__device__ __forceinline__ void stage_records(float2* dst, const float2* __restrict__ src, int n)
{
    float4* d4 = reinterpret_cast<float4*>(dst);
    const float4* s4 = reinterpret_cast<const float4*>(src);
    for (int i = threadIdx.x; i < n / 2; i += THREADS) cp_async16(d4 + i, s4 + i);
}

// Staging by the CTA's threads: the SM streams nothing while a CTA copies
// (other CTAs on the SM, if any, keep streaming).  MODE 0: stage the pieces
// the plan marks; MODE 1: no record staging, every piece reads its records
// through L1.  D > 0: the queries stream through a D-slot cp.async ring
// placed after the p.buf_stride staged records.
template <int THREADS, int MINB, int U, int MODE, int D>
__global__ void __launch_bounds__(THREADS, MINB) batch_eval_kernel(const EvalParams p, const float* x, float* y)
{
    extern __shared__ __align__(16) float2 s_idx[];
    __shared__ int s_next;
    float4* ring = reinterpret_cast<float4*>(s_idx + (MODE == 0 ? p.buf_stride : 0));
    int staged_f = -1;
    // the CTA's own range first, then unclaimed ones in order: the cost model
    // balances the ranges, the counter absorbs what it misjudges
    for (int rg = blockIdx.x; rg < p.n_ranges;) {
    const int it1 = p.range[rg + 1];
    for (int it = p.range[rg]; it < it1; ++it) {
        const WorkItem w = p.items[it];
        const BatchFunc& g = p.bf[w.f];
        if (MODE == 0 && w.staged) {
            if (staged_f != w.f) {
                __syncthreads();  // nobody reads the previous function's records any more
                stage_records<THREADS>(s_idx, p.recP + g.poff, g.K);
                stage_records<THREADS>(s_idx + g.K, p.recS + 2 * g.koff, 2 * (g.N + 1));
                cp_async_commit();
                cp_async_wait<0>();
                __syncthreads();
                staged_f = w.f;
            }
            run_piece<U, D, true>(p, g, w, s_idx, x, y, ring);
        } else {
            run_piece<U, D, false>(p, g, w, nullptr, x, y, ring);
        }
    }
    __syncthreads();  // every thread has read the previous s_next
    if (threadIdx.x == 0) s_next = (int)gridDim.x + atomicAdd(p.counter, 1);
    __syncthreads();
    rg = s_next;
    }
}

// Asynchronous staging, one CTA per SM with two record buffers: while the
// CTA streams the queries of one piece, a bulk copy (cp.async.bulk, the 1-D
// TMA form) brings the next staged piece's records into the other buffer,
// so the SM keeps streaming through the copy.  Every wait is bounded: on a
// timeout the CTA records it in *status, waits (bounded) for its copies in
// flight and stops.
// Failure injection (p.withheld = 1): each staging barrier expects one
// arrival more than the kernel makes, so no wait can succeed and the first
// one runs out after p.wait_ns; after the timeout thread 0 makes the
// withheld arrival, and the final waits then complete exactly when the
// bulk copies have landed, so that no copy is in flight when the CTA exits.
template <int U>
__global__ void __launch_bounds__(1024, 1) batch_eval_async_kernel(const EvalParams p, const float* x, float* y)
{
    extern __shared__ __align__(16) float2 s_idx[];
    __shared__ __align__(8) uint64_t s_bar[2];
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1 + p.withheld);
        mbar_init(&s_bar[1], 1 + p.withheld);
        fence_mbar_init();
    }
    __syncthreads();
    // buffer bookkeeping, identical in every thread
    int hold[2] = {-1, -1};          // function whose records the buffer holds or receives
    uint32_t parity[2] = {0u, 0u};   // parity of the buffer's next completion
    bool busy[2] = {false, false};   // a copy into the buffer has not been waited for
    bool failed = false;
    auto issue = [&](int bi, int f) {
        if (threadIdx.x == 0) {
            const BatchFunc& g = p.bf[f];
            const uint32_t bytesP = 8u * (uint32_t)g.K, bytesS = 16u * (uint32_t)(g.N + 1);
            float2* dst = s_idx + (size_t)bi * p.buf_stride;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&s_bar[bi], bytesP + bytesS);
            bulk_copy_g2s(dst, p.recP + g.poff, bytesP, &s_bar[bi]);
            bulk_copy_g2s(dst + g.K, p.recS + 2 * g.koff, bytesS, &s_bar[bi]);
        }
        hold[bi] = f;
        busy[bi] = true;
    };
    auto wait = [&](int bi) {
        const bool ok = mbar_wait_bounded(&s_bar[bi], parity[bi], p.wait_ns);
        if (ok) {  // a copy that did not complete stays busy for the final wait
            parity[bi] ^= 1u;
            busy[bi] = false;
        }
        return ok;
    };
    const int it0 = p.range[blockIdx.x], it1 = p.range[blockIdx.x + 1];
    for (int it = it0; it < it1; ++it) {
        const WorkItem w = p.items[it];
        __syncthreads();  // every thread is done with the previous piece's buffer
        int bi = -1;
        if (w.staged) {
            bi = hold[0] == w.f ? 0 : (hold[1] == w.f ? 1 : -1);
            if (bi < 0) {
                // no copy of this function in flight (a prefetch would have been
                // for it), so at most one buffer is busy
                bi = busy[0] ? 1 : 0;
                if (busy[bi] && !wait(bi))
                    failed = true;
                else
                    issue(bi, w.f);
            }
        }
        if (it + 1 < it1) {
            const WorkItem nx = p.items[it + 1];
            if (nx.staged && hold[0] != nx.f && hold[1] != nx.f) {
                const int ob = bi >= 0 ? (bi ^ 1) : (busy[0] ? 1 : 0);
                if (!busy[ob]) issue(ob, nx.f);
            }
        }
        if (bi >= 0 && busy[bi] && hold[bi] == w.f && !wait(bi)) failed = true;
        if (__syncthreads_or(failed)) {
            failed = true;
            break;
        }
        const BatchFunc& g = p.bf[w.f];
        if (bi >= 0)
            run_staged<U>(p, g, w, s_idx + (size_t)bi * p.buf_stride, x, y);
        else
            run_direct<U>(p, g, w, x, y);
    }
    // copies still in flight (only after a failed wait): wait for them, bounded
    // (busy[] and failed are the same in every thread)
    if (failed && p.withheld) {
        if (threadIdx.x == 0)
            for (int b = 0; b < 2; ++b)
                if (busy[b]) mbar_arrive(&s_bar[b]);
        __syncthreads();
    }
    for (int b = 0; b < 2; ++b)
        if (busy[b]) wait(b);
    if (failed && threadIdx.x == 0) atomicOr(p.status, 4);
}

// Launch shapes the planner and the autotuner choose from.  All keep <= 64
// registers per thread (1024 threads per SM).  A shape stages a function's
// index only if it fits the shape's staging budget: the shared memory one of
// its CTAs gets (ctas per SM) minus the ring.
using BatchEvalKernel = void (*)(const EvalParams, const float*, float*);
enum StageKind { kStageAsync = 0, kStageSync = 1, kStageNone = 2 };
constexpr int kRingDepth = 4;
constexpr int kRangesPerCta = 3;  // cost-balanced ranges per CTA of a dynamic shape
struct EvalShape {
    int threads;
    int ctas;   // CTAs per SM the shape is meant to run
    int stage;  // StageKind
    int ring;   // cp.async ring depth (0: vectors in registers)
    BatchEvalKernel kern;
};
const EvalShape kShapes[] = {
    // 1 CTA / SM, records staged by the CTA (up to all of its shared memory),
    // 4 query vectors in registers
    {1024, 1, kStageSync, 0, batch_eval_kernel<1024, 1, 4, 0, 0>},
    // 1 CTA / SM, records staged by the CTA, queries through a 4-slot ring
    {1024, 1, kStageSync, kRingDepth, batch_eval_kernel<1024, 1, 4, 0, kRingDepth>},
    // 2 CTAs / SM, records staged by the CTA, 4 vectors in registers
    {512, 2, kStageSync, 0, batch_eval_kernel<512, 2, 4, 0, 0>},
    // 1 CTA / SM, records through L1, queries through a 4-slot ring
    {1024, 1, kStageNone, kRingDepth, batch_eval_kernel<1024, 1, 4, 1, kRingDepth>},
    // 1 CTA / SM, two record buffers filled by bulk copies, 4 vectors in registers
    {1024, 1, kStageAsync, 0, batch_eval_async_kernel<4>},
};
constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

}  // namespace pwl

using namespace pwl;

struct pwl_batch_s {
    int device;
    int64_t F;
    int kinds;                  // kKindsAnalytic | kKindsSampled of the functions
    int64_t m_per;
    std::vector<int64_t> N;     // intervals per function
    std::vector<int64_t> koff;  // knot offsets
    std::vector<int64_t> K;     // cells per function
    int64_t total_knots, total_cells_design, total_chunks, total_cells_index;
    size_t index_budget;        // shared memory a staged index may take
    void* dev;                  // one allocation for everything below
    pwl_func* funcs;
    int64_t *d_koff, *d_moff, *d_choff;
    double* knots;
    double* values;
    void* design_scratch;
    void* project_scratch;
    BatchFunc* bf;
    float *xk, *vk, *slope;
    int* cj;
    float2 *recP, *recS;
    int* status;                // device word: bit 2 = an evaluation wait timed out
    int* order;                 // functions by decreasing density cells (design order)
    // evaluation plan
    std::vector<int64_t> qoff;  // query offsets of the plan
    void* plan_dev;             // items, then the CTA ranges
    WorkItem* items;
    int* range;
    int* counter;               // next dynamic range, zeroed before each launch
    int n_ranges;
    int grid;
    int shape;
    int64_t stage_min;          // stage when queries * stage_min >= index bytes
    size_t smem;
    int buf_stride;             // float2 records per staging buffer
    int64_t n_items, n_staged;
    int64_t total_queries;
    bool planned;
    uint64_t wait_ns;           // limit of one wait for a staging copy (kWaitLimitNs unless a test sets it)
    int withheld;               // failure injection of pwl_batch_inject_wait_timeout
};

namespace {

void batch_free(pwl_batch b)
{
    if (!b) return;
    if (b->plan_dev) cudaFree(b->plan_dev);
    if (b->dev) cudaFree(b->dev);
    delete b;
}

size_t index_bytes(const pwl_batch_s* b, int64_t f)
{
    return 8 * (size_t)b->K[f] + 16 * (size_t)(b->N[f] + 1);
}

// Cut the concatenated query stream into G contiguous ranges of about equal
// cost and mark which pieces stage their index.  The cost of a piece, in
// bytes of HBM-rate streaming: 8 per query (x in, y out; kDirectQueryCost
// when the records are read through L1 instead of shared memory), the index
// bytes when the piece stages its function's index, and kPieceCost for the
// fixed latency of starting a piece.  Each CTA's target is the cost still
// unassigned divided by the CTAs still open, so that a CTA that closes
// short or long does not push the difference onto the last one.
constexpr double kPieceCost = 65536.0;
constexpr double kQueryCost = 8.0;
constexpr double kDirectQueryCost = 24.0;

void make_plan(const pwl_batch_s* b, const int64_t* qo, int G, int64_t stage_min, size_t budget,
               std::vector<WorkItem>& items, std::vector<int>& range)
{
    auto staged_piece = [&](int64_t f, int64_t nq) {
        const size_t ib = index_bytes(b, f);
        return stage_min > 0 && ib <= budget && (size_t)nq * (size_t)stage_min >= ib;
    };
    auto cost = [&](int64_t f, int64_t nq) {
        const bool st = staged_piece(f, nq);
        return kPieceCost + (st ? (double)index_bytes(b, f) + kQueryCost * (double)nq : kDirectQueryCost * (double)nq);
    };
    constexpr int64_t kMinPiece = 4096;      // no piece of a split function shorter than this
    constexpr int64_t kMaxPiece = 1LL << 30; // the evaluation loop indexes a piece with 32-bit ints
    double rest = 0;
    for (int64_t f = 0; f < b->F; ++f) {
        const int64_t nq = qo[f + 1] - qo[f];
        for (int64_t q = 0; q < nq; q += kMaxPiece) rest += cost(f, std::min(nq - q, kMaxPiece));
    }
    items.clear();
    range.assign(G + 1, 0);
    int cta = 0;
    double used = 0, target = rest / G;
    auto push = [&](int64_t f, int64_t q0, int64_t q1) {
        items.push_back(WorkItem{(int)f, staged_piece(f, q1 - q0) ? 1 : 0, q0, q1});
    };
    for (int64_t f = 0; f < b->F; ++f) {
        int64_t q = qo[f];
        const int64_t q1 = qo[f + 1];
        while (q < q1) {
            const int64_t nq = std::min(q1 - q, kMaxPiece);
            const double need = cost(f, nq);
            if (cta == G - 1 || used + need <= target) {
                push(f, q, q + nq);
                used += need;
                rest -= need;
                q += nq;
                continue;
            }
            // the piece does not fit: split it at the target, or give it to
            // whichever CTA it overshoots least
            const double avail = target - used;
            int64_t split = (int64_t)((avail - kPieceCost - (staged_piece(f, nq) ? (double)index_bytes(b, f) : 0.0)) /
                                      kQueryCost);
            split &= ~(int64_t)3;  // pieces keep the 16-byte boundaries of x and y
            if (split >= kMinPiece && nq - split >= kMinPiece) {
                push(f, q, q + split);
                const double c = cost(f, split);
                used += c;
                rest += cost(f, nq - split) - need;  // the remainder pays its own fixed costs
                q += split;
            } else if (avail >= 0.5 * need) {
                push(f, q, q + nq);
                used += need;
                rest -= need;
                q += nq;
            }
            range[++cta] = (int)items.size();
            used = 0;
            target = rest / (G - cta);
        }
    }
    while (cta < G) range[++cta] = (int)items.size();
}

}  // namespace

extern "C" {

pwl_status pwl_batch_create(const pwl_func* funcs, const int64_t* n_intervals, int64_t n_funcs,
                            int64_t m_per_interval, int64_t cells_per_knot, pwl_batch* out)
{
    clear_error();
    if (!out) return fail(PWL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!funcs || !n_intervals) return fail(PWL_EINVAL, "funcs / n_intervals is NULL");
    if (n_funcs < 1 || n_funcs > (1 << 20)) return fail(PWL_EINVAL, "n_funcs must be in [1, 2^20]");
    if (m_per_interval < 0 || m_per_interval > 4096) return fail(PWL_EINVAL, "m_per_interval must be in [0, 4096]");
    if (cells_per_knot < 0 || cells_per_knot > 64) return fail(PWL_EINVAL, "cells_per_knot must be in [0, 64]");
    const int64_t mper = m_per_interval > 0 ? m_per_interval : 64;
    const int64_t cpk = cells_per_knot > 0 ? cells_per_knot : 3;
    for (int64_t f = 0; f < n_funcs; ++f) {
        if (validate_func(funcs + f) != PWL_OK) return fail(PWL_EINVAL, "function %lld: %s", (long long)f,
                                                            pwl_last_error());
        if (n_intervals[f] < 1 || n_intervals[f] > kMaxBatchIntervals)
            return fail(PWL_EINVAL, "function %lld: n_intervals must be in [1, %d]", (long long)f,
                        kMaxBatchIntervals);
    }
    pwl_batch b = new (std::nothrow) pwl_batch_s();
    if (!b) return fail(PWL_ENOMEM, "host allocation failed");
    b->wait_ns = kWaitLimitNs;
    b->withheld = 0;
    cudaGetDevice(&b->device);
    const DeviceInfo& di = device_info();
    b->F = n_funcs;
    b->kinds = kinds_of(funcs, n_funcs);
    b->m_per = mper;
    b->N.assign(n_intervals, n_intervals + n_funcs);
    b->koff.resize(n_funcs + 1);
    b->K.resize(n_funcs);
    // the largest index one CTA can stage (shape 0: one CTA per SM)
    b->index_budget = di.smem_optin - 1024;
    std::vector<int64_t> moff(n_funcs + 1), choff(n_funcs + 1);
    std::vector<BatchFunc> bfh(n_funcs);
    b->koff[0] = moff[0] = choff[0] = 0;
    int64_t poff = 0, soff = 0;
    for (int64_t f = 0; f < n_funcs; ++f) {
        const int64_t N = b->N[f];
        b->koff[f + 1] = b->koff[f] + N + 1;
        moff[f + 1] = moff[f] + mper * N;
        choff[f + 1] = choff[f] + design_chunks(mper * N);
        // cells_per_knot cells per knot, fewer if the index would not fit the
        // budget (then more knots share cells); an index that cannot fit is
        // never staged and keeps cells_per_knot
        const int64_t room = ((int64_t)b->index_budget - 16 * (N + 1)) / 8;
        int64_t K = room >= 256 ? std::min<int64_t>(cpk * (N + 1), room) : cpk * (N + 1);
        K = std::max<int64_t>(2, K & ~(int64_t)1);  // even: the records of every function start 16-byte aligned
        b->K[f] = K;
        BatchFunc& d = bfh[f];
        memset(&d, 0, sizeof(d));
        d.koff = b->koff[f];
        d.soff = soff;
        d.poff = poff;
        d.N = (int)N;
        d.K = (int)K;
        poff += K;
        soff += N + 2;
    }
    // design order: the functions with the most density cells first, so that
    // the persistent design launch ends on small functions
    std::vector<int> order(n_funcs);
    for (int64_t f = 0; f < n_funcs; ++f) order[f] = (int)f;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->N[x] > b->N[y]; });
    b->total_knots = b->koff[n_funcs];
    b->total_cells_design = moff[n_funcs];
    b->total_chunks = choff[n_funcs];
    b->total_cells_index = poff;
    const size_t F = (size_t)n_funcs, T = (size_t)b->total_knots;
    const size_t sizes[] = {align256(sizeof(pwl_func) * F),
                            align256(8 * (F + 1)),
                            align256(8 * (F + 1)),
                            align256(8 * (F + 1)),
                            align256(8 * T),
                            align256(8 * T),
                            align256(design_scratch_bytes(n_funcs, b->total_cells_design, b->total_chunks)),
                            align256(project_scratch_bytes(b->total_knots, b->total_knots - n_funcs)),
                            align256(sizeof(BatchFunc) * F),
                            align256(4 * T),
                            align256(4 * T),
                            align256(4 * (size_t)soff),
                            align256(4 * T),
                            align256(8 * (size_t)poff),
                            align256(16 * T),
                            align256(sizeof(int)),
                            align256(sizeof(int) * F)};
    void** slots[] = {(void**)&b->funcs, (void**)&b->d_koff, (void**)&b->d_moff, (void**)&b->d_choff,
                      (void**)&b->knots, (void**)&b->values, &b->design_scratch, &b->project_scratch,
                      (void**)&b->bf, (void**)&b->xk, (void**)&b->vk, (void**)&b->slope, (void**)&b->cj,
                      (void**)&b->recP, (void**)&b->recS, (void**)&b->status, (void**)&b->order};
    static_assert(sizeof(sizes) / sizeof(sizes[0]) == sizeof(slots) / sizeof(slots[0]), "one size per slot");
    size_t total = 0;
    for (size_t s : sizes) total += s;
    cudaError_t e = dev_malloc(&b->dev, total);
    if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "cudaMalloc(batch)");
    }
    char* p = static_cast<char*>(b->dev);
    for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]); ++i) {
        *slots[i] = p;
        p += sizes[i];
    }
    if ((e = cudaMemcpy(b->funcs, funcs, sizeof(pwl_func) * F, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_koff, b->koff.data(), 8 * (F + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_moff, moff.data(), 8 * (F + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_choff, choff.data(), 8 * (F + 1), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->bf, bfh.data(), sizeof(BatchFunc) * F, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(b->status, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMemcpy(b->order, order.data(), sizeof(int) * F, cudaMemcpyHostToDevice)) != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch upload");
    }
    b->shape = 0;
    b->stage_min = 16;
    *out = b;
    return PWL_OK;
}

pwl_status pwl_batch_destroy(pwl_batch b)
{
    clear_error();
    batch_free(b);
    return PWL_OK;
}

pwl_status pwl_batch_design(pwl_batch b, int32_t precision, void* stream)
{
    clear_error();
    if (!b) return fail(PWL_EINVAL, "batch is NULL");
    if (precision != PWL_PREC_FP64 && precision != PWL_PREC_FP32) return fail(PWL_EINVAL, "unknown precision");
    DesignPlan p{};
    p.F = (int)b->F;
    p.precision = precision;
    p.kinds = b->kinds;
    p.funcs = b->funcs;
    p.koff = b->d_koff;
    p.moff = b->d_moff;
    p.choff = b->d_choff;
    p.total_knots = b->total_knots;
    p.total_cells = b->total_cells_design;
    p.total_chunks = b->total_chunks;
    p.knots = b->knots;
    design_carve_scratch(p, b->design_scratch);
    p.order = b->order;
    // the fused path keeps no cumulative values: its per-chunk markers use that
    // area, and its FP32 mode keeps the FP32 densities in the density area
    p.clast = reinterpret_cast<int*>(p.G);
    return design_fused_launch(p, as_stream(stream));
}

pwl_status pwl_batch_project(pwl_batch b, int32_t form, int32_t quad_points, int32_t precision, void* stream)
{
    clear_error();
    if (!b) return fail(PWL_EINVAL, "batch is NULL");
    if (form != PWL_INTERP && form != PWL_PROJECT) return fail(PWL_EINVAL, "unknown form %d", form);
    if (quad_points == 0) quad_points = 8;
    if (quad_points < 1 || quad_points > 16) return fail(PWL_EINVAL, "quad_points must be in [1, 16]");
    if (precision != PWL_PREC_FP64 && precision != PWL_PREC_FP32) return fail(PWL_EINVAL, "unknown precision");
    ProjectPlan p{};
    p.F = (int)b->F;
    p.precision = precision;
    p.kinds = b->kinds;
    p.form = form;
    p.max_rows = (int)(*std::max_element(b->N.begin(), b->N.end()) + 1);
    p.total_knots = b->total_knots;
    p.total_intervals = b->total_knots - b->F;
    p.funcs = b->funcs;
    p.koff = b->d_koff;
    p.knots = b->knots;
    p.values = b->values;
    project_carve_scratch(p, b->project_scratch);
    // many functions: one warp each (partitioned Thomas); few: one CTA each
    // (cyclic reduction)
    p.solver = b->F >= 64 ? 1 : 0;
    p.order = b->order;
    return project_launch(p, gauss_legendre_rule(quad_points), as_stream(stream));
}

pwl_status pwl_batch_build(pwl_batch b, void* stream)
{
    clear_error();
    if (!b) return fail(PWL_EINVAL, "batch is NULL");
    const int grid = (int)std::min<int64_t>(b->F, (int64_t)device_info().sms * 2);
    batch_index_kernel<<<grid, kIndexThreads, 0, as_stream(stream)>>>((int)b->F, b->knots, b->values, b->bf, b->xk,
                                                                      b->vk, b->slope, b->cj, b->recP, b->recS);
    PWL_CHECK_LAUNCH("batch_index_kernel");
    return PWL_OK;
}

pwl_status pwl_batch_check(pwl_batch b, void* stream)
{
    clear_error();
    if (!b) return fail(PWL_EINVAL, "batch is NULL");
    std::vector<BatchFunc> h(b->F);
    int status = 0;
    cudaStream_t s = as_stream(stream);
    PWL_CUDA_TRY(cudaMemcpyAsync(h.data(), b->bf, sizeof(BatchFunc) * b->F, cudaMemcpyDeviceToHost, s));
    PWL_CUDA_TRY(cudaMemcpyAsync(&status, b->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    PWL_CUDA_TRY(cudaMemsetAsync(b->status, 0, sizeof(int), s));
    PWL_CUDA_TRY(cudaStreamSynchronize(s));
    if (status & 4) return fail(PWL_ETIMEOUT, "an evaluation launch gave up waiting for a staging copy");
    for (int64_t f = 0; f < b->F; ++f) {
        if (h[f].status & 2) return fail(PWL_EINVAL, "function %lld: a knot or value is not finite", (long long)f);
        if (h[f].status & 1)
            return fail(PWL_EINVAL, "function %lld: knots not strictly increasing in FP32", (long long)f);
    }
    return PWL_OK;
}

pwl_status pwl_batch_plan(pwl_batch b, const int64_t* query_offsets, int32_t shape, int64_t stage_min)
{
    clear_error();
    if (!b) return fail(PWL_EINVAL, "batch is NULL");
    if (!query_offsets) return fail(PWL_EINVAL, "query_offsets is NULL");
    if (query_offsets[0] != 0) return fail(PWL_EINVAL, "query_offsets[0] must be 0");
    for (int64_t f = 0; f < b->F; ++f)
        if (query_offsets[f + 1] < query_offsets[f]) return fail(PWL_EINVAL, "query_offsets must be non-decreasing");
    if (shape < -1 || shape >= kNumShapes) return fail(PWL_EINVAL, "shape must be in [-1, %d]", kNumShapes - 1);
    if (stage_min < -1) return fail(PWL_EINVAL, "stage_min must be >= -1");
    if (shape < 0) shape = b->shape;
    if (stage_min < 0) stage_min = b->stage_min;
    const EvalShape& sh = kShapes[shape];
    if (sh.stage == kStageNone) stage_min = 0;
    // staging budget of one buffer: the CTA's share of the SM's shared memory
    // minus the ring (and halved for two buffers)
    const DeviceInfo& di = device_info();
    const size_t ring = (size_t)sh.ring * 16 * (size_t)sh.threads;
    const size_t cta_smem = std::min(di.smem_optin, di.smem_per_sm / (size_t)sh.ctas - 1024);
    size_t budget = cta_smem > ring + 1024 ? cta_smem - ring - 1024 : 0;
    if (sh.stage == kStageAsync) budget /= 2;
    if (sh.stage == kStageNone) budget = 0;
    budget &= ~(size_t)15;
    size_t buf = 0;  // bytes of the largest index that may be staged
    for (int64_t f = 0; f < b->F; ++f) {
        const size_t ib = index_bytes(b, f);
        if (ib <= budget) buf = std::max(buf, ib);
    }
    buf = (buf + 15) & ~(size_t)15;
    const size_t smem = (sh.stage == kStageAsync ? 2 * buf : (sh.stage == kStageSync ? buf : 0)) + ring;
    int grid = 0;
    PWL_CUDA_TRY(occupancy_grid(sh.kern, sh.threads, smem, &grid));
    // ranges per CTA: several (taken dynamically after the first) except for
    // the asynchronous shape, whose prefetch looks ahead inside one range
    const int n_ranges = sh.stage == kStageAsync ? grid : grid * kRangesPerCta;
    std::vector<WorkItem> items;
    std::vector<int> range;
    make_plan(b, query_offsets, n_ranges, stage_min, budget, items, range);
    void* dev = nullptr;
    const size_t bytes_items = align256(sizeof(WorkItem) * std::max<size_t>(items.size(), 1));
    const size_t bytes_range = align256(sizeof(int) * (size_t)(n_ranges + 1));
    PWL_CUDA_TRY(dev_malloc(&dev, bytes_items + bytes_range + sizeof(int)));
    cudaError_t e = cudaSuccess;
    if (!items.empty()) e = cudaMemcpy(dev, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(static_cast<char*>(dev) + bytes_items, range.data(), sizeof(int) * (size_t)(n_ranges + 1),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dev);
        return cuda_fail(e, "batch plan upload");
    }
    if (b->plan_dev) cudaFree(b->plan_dev);
    b->plan_dev = dev;
    b->items = static_cast<WorkItem*>(dev);
    b->range = reinterpret_cast<int*>(static_cast<char*>(dev) + bytes_items);
    b->counter = reinterpret_cast<int*>(static_cast<char*>(dev) + bytes_items + bytes_range);
    b->n_ranges = n_ranges;
    b->grid = grid;
    b->shape = shape;
    b->stage_min = stage_min;
    b->smem = smem;
    b->buf_stride = (int)(buf / sizeof(float2));
    b->n_items = (int64_t)items.size();
    b->n_staged = 0;
    for (const WorkItem& w : items) b->n_staged += w.staged;
    b->qoff.assign(query_offsets, query_offsets + b->F + 1);
    b->total_queries = query_offsets[b->F];
    b->planned = true;
    return PWL_OK;
}

pwl_status pwl_batch_eval(pwl_batch b, const float* d_x, float* d_y, void* stream)
{
    clear_error();
    if (!b) return fail(PWL_EINVAL, "batch is NULL");
    if (!b->planned) return fail(PWL_EINVAL, "pwl_batch_plan has not been called");
    if (b->total_queries == 0) return PWL_OK;
    if (!d_x || !d_y) return fail(PWL_EINVAL, "x / y is NULL");
    if ((reinterpret_cast<uintptr_t>(d_x) | reinterpret_cast<uintptr_t>(d_y)) % 16 != 0)
        return fail(PWL_EINVAL, "x and y must be 16-byte aligned");
    const EvalShape& sh = kShapes[b->shape];
    PWL_CUDA_TRY(raise_smem_limit(sh.kern, b->smem));
    const EvalParams p{b->items, b->range, b->n_ranges, b->counter, b->bf, b->xk, b->recP, b->recS,
                       b->buf_stride, b->status, b->wait_ns, b->withheld};
    if (sh.stage != kStageAsync)
        PWL_CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(int), as_stream(stream)));
    sh.kern<<<b->grid, sh.threads, b->smem, as_stream(stream)>>>(p, d_x, d_y);
    PWL_CHECK_LAUNCH("batch_eval_kernel");
    return PWL_OK;
}

pwl_status pwl_batch_autotune(pwl_batch b, const float* d_x, float* d_y, int32_t reps, float* timings_ms,
                              void* stream)
{
    clear_error();
    if (!b) return fail(PWL_EINVAL, "batch is NULL");
    if (!b->planned) return fail(PWL_EINVAL, "pwl_batch_plan has not been called");
    if (reps < 1 || reps > 100) return fail(PWL_EINVAL, "reps must be in [1, 100]");
    const std::vector<int64_t> qo = b->qoff;
    const int64_t stage_opts[] = {0, 4, 16, 64};
    cudaStream_t s = as_stream(stream);
    cudaEvent_t e0, e1;
    PWL_CUDA_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(PWL_ECUDA, "cudaEventCreate");
    }
    float best = 3.0e38f;
    int best_shape = b->shape;
    int64_t best_stage = b->stage_min;
    pwl_status st = PWL_OK;
    constexpr int kStageOpts = sizeof(stage_opts) / sizeof(stage_opts[0]);
    for (int sh = 0; sh < kNumShapes && st == PWL_OK; ++sh) {
        for (int si = 0; si < kStageOpts; ++si) {
            const int64_t sm = stage_opts[si];
            if (kShapes[sh].stage == kStageNone && si > 0) {  // stage_min has no effect: one timing
                if (timings_ms) timings_ms[sh * kStageOpts + si] = timings_ms[sh * kStageOpts];
                continue;
            }
            if ((st = pwl_batch_plan(b, qo.data(), sh, sm)) != PWL_OK) break;
            if ((st = pwl_batch_eval(b, d_x, d_y, stream)) != PWL_OK) break;  // warm-up
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && st == PWL_OK; ++r) st = pwl_batch_eval(b, d_x, d_y, stream);
            cudaEventRecord(e1, s);
            if (st != PWL_OK) break;
            const cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "autotune timing");
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)reps;
            if (timings_ms) timings_ms[sh * kStageOpts + si] = ms;
            if (ms < best) {
                best = ms;
                best_shape = sh;
                best_stage = sm;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PWL_OK) return st;
    return pwl_batch_plan(b, qo.data(), best_shape, best_stage);
}

pwl_status pwl_batch_inject_wait_timeout(pwl_batch b, int32_t withhold, uint64_t wait_limit_ns)
{
    clear_error();
    if (!b) return fail(PWL_EINVAL, "batch is NULL");
    if (withhold != 0 && withhold != 1) return fail(PWL_EINVAL, "withhold must be 0 or 1");
    if (wait_limit_ns > kWaitLimitNs) return fail(PWL_EINVAL, "wait limit above %llu ns", (unsigned long long)kWaitLimitNs);
    b->withheld = withhold;
    b->wait_ns = wait_limit_ns ? wait_limit_ns : kWaitLimitNs;
    return PWL_OK;
}

pwl_status pwl_batch_get_info(pwl_batch b, pwl_batch_info* info)
{
    clear_error();
    if (!b || !info) return fail(PWL_EINVAL, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->n_funcs = b->F;
    info->total_knots = b->total_knots;
    info->total_cells = b->total_cells_index;
    info->index_bytes = 8 * b->total_cells_index + 16 * b->total_knots;
    info->total_queries = b->planned ? b->total_queries : 0;
    info->eval_grid = b->planned ? b->grid : 0;
    info->eval_threads = kShapes[b->shape].threads;
    info->eval_shape = b->shape;
    info->n_items = b->planned ? b->n_items : 0;
    info->n_staged = b->planned ? b->n_staged : 0;
    info->stage_min = b->stage_min;
    info->smem_bytes = b->planned ? (int64_t)b->smem : 0;
    info->d_knot_offsets = b->d_koff;
    info->d_knots = b->knots;
    info->d_values = b->values;
    info->d_knots_fp32 = b->xk;
    info->d_values_fp32 = b->vk;
    return PWL_OK;
}

}  // extern "C"
