// pwl_eval.cu -- CPWL evaluation (Algorithm 1) over a query stream.
//
// Main path (pwl_eval): a persistent grid; every CTA stages a cell index
// (8-byte cell records and the side records of the knots) in shared memory,
// then streams 16-byte vectors of queries with several loads in flight per
// thread.  Per query: clamp to [x_0, x_N]; one fma and a
// truncation give the cell (step 1 of Algorithm 1 becomes a lookup); one
// 8-byte shared-memory load gives the cell's line, y = y_c + (x - x_c) s
// (steps 2-3 fused into one FMA).  Only queries whose cell holds a knot load
// a second 8-byte side record, {v_k, s} for their side of the knot; several
// knots in one cell (rare: the cells are narrower than most intervals) are
// walked through the FP32 knot array.
//
// Tables whose 8-byte index would not leave room for two CTAs per SM use the
// 16-byte index instead (one record {x_j, v_j, s_j, s_{j+1}} per cell, one
// 16-byte load per query): fewer instructions, more shared-memory wavefronts.
//
// Comparison paths (pwl_eval_variant, and pwl_eval_synthetic_variant with
// queries generated in registers):
//   mode 0  the paper's Algorithm 1 with its search (Section IV): a binary
//           search over the FP32 knots in shared memory, unrolled for the
//           table's size and made of selects (no divergent branches), delta
//           by a division, (1 - delta) v_{i-1} + delta v_i
//   mode 1  interval lookup through the 16-byte index, then the texture
//           unit's linear filter at i - 1 + delta + 1/2 (Section IV-B)
//   mode 2, 3  the main path forced to the 8-byte or the 16-byte index
//   mode 6  the main path forced to the 8-byte index with one side record
//           per knot
//   mode 4  the search of mode 0, then the texture filter (the paper's
//           "optimized partition, hardware interpolation", Table I)
//   mode 5  uniform partition: no search, the texture coordinate
//           (x - x_0) N / (x_N - x_0) + 1/2 (Section IV's O(1) case with
//           hardware interpolation, Table I); exact only for a table whose
//           knots are uniform
#include <math.h>

#include <algorithm>

#include "pwl_stream.cuh"
#include "pwl_table.cuh"

namespace pwl {

namespace {

constexpr int kUnroll = 4;

struct EvalArgs {
    const float2* recP;   // 8-byte layout: K cell records
    const float2* recS;   // 8-byte layout: 2 (N+1) side records
    const float2* recS8;  // 8-byte layout with one side record per knot: N+1 records {v_k, s_{k+1}}
    const float* xk;      // N+1 FP32 knots (chain walks of the 8-byte layout)
    const float4* rec16;  // 16-byte layout: K cell records + chain area
    const TableHeader* hdr;
    int K, N;
    int s_staged;         // 8-byte layout: side records in shared memory (else global)
    int n_smem;           // 16-byte layout: records staged (at launch: the room reserved)
    int max_chain;        // set from the device header by the kernel
    float a, b, inv_w, off, w;
    int64_t head;         // scalar queries before the first 16-byte boundary of x
    int64_t nvec;         // 16-byte vectors after the head
};

// 8-byte layout.  Branch-free apart from chains: every lane computes its
// cell anchor, knot lanes additionally load their side record (a predicated
// load), and one FMA finishes.
// A cell holding several knots: from its first knot k (at xk) to the last
// knot <= xc, reading the knots from global memory.  Called out of line
// (one CTA per SM), so that the lookup of the (many) queries in cells
// without a chain keeps the instruction schedule of a chain-free table.
__device__ __noinline__ int2 walk_chain8(float xc, int k, float xk, const float* __restrict__ xkg, int max_chain,
                                         int N)
{
    for (int g = 0; g < max_chain && k < N; ++g) {
        const float xn = __ldg(xkg + k + 1);
        if (!(xc >= xn)) break;
        ++k;
        xk = xn;
    }
    return make_int2(k, __float_as_int(xk));
}

// SIDE8: one side record per knot, {v_k, s_{k+1}}; left of x_k the slope is
// s_k, from the record of knot k - 1 (the same v_k + (x - x_k) s as the two
// side records give, at half their shared memory).
template <bool CHAINS, bool OUTLINE = false, bool SIDE8 = false>
struct Lerp8 {
    const float2* sP;
    const float2* sS;
    const EvalArgs& p;
    __device__ __forceinline__ float operator()(float x) const
    {
        const float xc = clamp_nan(x, p.a, p.b);
        float cf;
        const int c = cell_of_f(xc, p.inv_w, p.off, p.K, cf);
        const float2 r = sP[c];
        const uint32_t bits = __float_as_uint(r.x);
        float anchor = __fmaf_rn(cf, p.w, p.a);
        float2 q = r;  // no knot in the cell: the cell's line {y_c, s} anchored at x_c
        if ((bits & 0xFFC00000u) == kLinkTag) {
            int k = (int)(bits & kKnotTagMask);
            float xk = r.y;
            if (CHAINS && (bits & kKnotTagChain)) {
                if (OUTLINE) {
                    const int2 w = walk_chain8(xc, k, xk, p.xk, p.max_chain, p.N);
                    k = w.x;
                    xk = __int_as_float(w.y);
                } else {
                    for (int g = 0; g < p.max_chain && k < p.N; ++g) {
                        const float xn = __ldg(p.xk + k + 1);
                        if (!(xc >= xn)) break;
                        ++k;
                        xk = xn;
                    }
                }
            }
            // x == x_k takes the right side: v_k + 0 * s is exactly v_k
            if constexpr (SIDE8) {
                q = sS[k];
                if (xc < xk) q.y = sS[k - 1].y;  // left of x_k (k >= 1 there: x >= x_0)
            } else {
                const int si = 2 * k + (xc >= xk ? 1 : 0);
                q = p.s_staged ? sS[si] : __ldg(p.recS + si);
            }
            anchor = xk;
        }
        return __fmaf_rn(xc - anchor, q.y, q.x);
    }
};

// 16-byte layout: one record {x_j, v_j, s_j, s_{j+1} | link} per cell.
template <bool CHAINS>
struct Lerp16 {
    const float4* s16;
    const EvalArgs& p;
    __device__ __forceinline__ float operator()(float x) const
    {
        const float xc = clamp_nan(x, p.a, p.b);
        const int c = cell_of(xc, p.inv_w, p.off, p.K);
        float4 r = s16[c];
        if (CHAINS) {
            for (int g = 0; g < p.max_chain && xc > r.x && is_link(r.w); ++g) {
                const int j = link_index(r.w);
                r = (j < p.n_smem) ? s16[j] : __ldg(p.rec16 + j);
            }
        }
        // x == x_j takes the left slope: v_j + 0 * s_j is exactly v_j
        const float s = (xc <= r.x) ? r.z : r.w;
        return __fmaf_rn(xc - r.x, s, r.y);
    }
};

template <typename IO, int U, class L>
__device__ __forceinline__ void eval_body(const EvalArgs& p, const L& f, const IO* x, IO* y, int64_t m)
{
    stream_body<IO, U>(p.head, p.nvec, f, x, y, m);
}

// LAYOUT 0: 8-byte index; 1: 16-byte index; 2: 8-byte index with one side
// record per knot.  MINB = 2 asks for <= 32
// registers so that two 1024-thread CTAs fit an SM (used when two copies of
// the index fit its shared memory); it keeps two 16-byte vectors in flight
// per thread instead of four, the same bytes in flight per SM.
template <typename IO, int LAYOUT, int MINB>
__global__ void __launch_bounds__(1024, MINB) eval_kernel(const EvalArgs args, const IO* x, IO* y, int64_t m)
{
    constexpr int U = (MINB >= 2) ? kUnroll / 2 : kUnroll;
    extern __shared__ float4 s_fwd[];
    EvalArgs p = args;
    if (LAYOUT == 0 || LAYOUT == 2) {
        float2* sP = reinterpret_cast<float2*>(s_fwd);
        float2* sS = sP + p.K;
        const int n_chain = p.hdr->n_chain_f;
        p.max_chain = p.hdr->max_chain_f;
        for (int i = threadIdx.x; i < p.K; i += blockDim.x) sP[i] = __ldg(p.recP + i);
        if (LAYOUT == 2)
            for (int i = threadIdx.x; i <= p.N; i += blockDim.x) sS[i] = __ldg(p.recS8 + i);
        else if (p.s_staged)
            for (int i = threadIdx.x; i < 2 * (p.N + 1); i += blockDim.x) sS[i] = __ldg(p.recS + i);
        __syncthreads();
        // the chain walk out of line where the registers allow the call (one
        // CTA per SM); inline at two CTAs per SM (32 registers a thread)
        constexpr bool S8 = LAYOUT == 2;
        if (n_chain == 0)
            eval_body<IO, U>(p, Lerp8<false, false, S8>{sP, sS, p}, x, y, m);
        else
            eval_body<IO, U>(p, Lerp8<true, MINB == 1, S8>{sP, sS, p}, x, y, m);
    } else {
        const int n_chain = p.hdr->n_chain_b;
        p.max_chain = p.hdr->max_chain_b;
        p.n_smem = min(p.K + n_chain, p.n_smem);  // the rest of the chain area stays in global memory
        for (int i = threadIdx.x; i < p.n_smem; i += blockDim.x) s_fwd[i] = __ldg(p.rec16 + i);
        __syncthreads();
        if (n_chain == 0)
            eval_body<IO, U>(p, Lerp16<false>{s_fwd, p}, x, y, m);
        else
            eval_body<IO, U>(p, Lerp16<true>{s_fwd, p}, x, y, m);
    }
}

// ---- compute ceiling: queries generated in registers (pwl_stream.cuh) ------
// Algorithm 1 on m generated queries: no query loaded, no result stored;
// every CTA adds the sum of its results to *sum (FP64).  The staging and the
// lookup are those of eval_kernel.
template <int LAYOUT, int MINB>
__global__ void __launch_bounds__(1024, MINB) eval_synth_kernel(const EvalArgs args, uint32_t seed, int64_t m,
                                                                double* sum)
{
    extern __shared__ float4 s_fwd[];
    EvalArgs p = args;
    const float w = __fsub_rn(p.b, p.a);
    float acc;
    if (LAYOUT == 0 || LAYOUT == 2) {
        float2* sP = reinterpret_cast<float2*>(s_fwd);
        float2* sS = sP + p.K;
        const int n_chain = p.hdr->n_chain_f;
        p.max_chain = p.hdr->max_chain_f;
        for (int i = threadIdx.x; i < p.K; i += blockDim.x) sP[i] = __ldg(p.recP + i);
        if (LAYOUT == 2)
            for (int i = threadIdx.x; i <= p.N; i += blockDim.x) sS[i] = __ldg(p.recS8 + i);
        else if (p.s_staged)
            for (int i = threadIdx.x; i < 2 * (p.N + 1); i += blockDim.x) sS[i] = __ldg(p.recS + i);
        __syncthreads();
        constexpr bool S8 = LAYOUT == 2;
        acc = n_chain == 0 ? synth_sum(Lerp8<false, false, S8>{sP, sS, p}, seed, p.a, w, m)
                           : synth_sum(Lerp8<true, false, S8>{sP, sS, p}, seed, p.a, w, m);
    } else {
        const int n_chain = p.hdr->n_chain_b;
        p.max_chain = p.hdr->max_chain_b;
        p.n_smem = min(p.K + n_chain, p.n_smem);
        for (int i = threadIdx.x; i < p.n_smem; i += blockDim.x) s_fwd[i] = __ldg(p.rec16 + i);
        __syncthreads();
        acc = n_chain == 0 ? synth_sum(Lerp16<false>{s_fwd, p}, seed, p.a, w, m)
                           : synth_sum(Lerp16<true>{s_fwd, p}, seed, p.a, w, m);
    }
    // the index may fill all of the shared memory: once every lookup is
    // done, its first 32 words hold the warp sums
    cta_sum_to(acc, reinterpret_cast<float*>(s_fwd), sum);
}

// ---- comparison paths (modes 0, 1, 4, 5) -----------------------------------
// Every variant kernel runs either on a query stream (SYNTH = false: x -> y
// with the streaming shape of pwl_eval) or on register-generated queries
// (SYNTH = true: the sum of the results goes to *sum).
struct StreamIO {
    const float* x;
    float* y;
    int64_t m;
    int64_t head, nvec;  // stream split (SYNTH = false)
    uint32_t seed;       // query generator (SYNTH = true)
    double* sum;
};

constexpr int kVarUnroll = 4;

// s_red: 32 floats of shared memory free once every lookup is done
template <bool SYNTH, class F>
__device__ __forceinline__ void run_variant(const StreamIO& io, const F& f, float a, float b, float* s_red)
{
    if constexpr (SYNTH)
        cta_sum_to(synth_sum(f, io.seed, a, __fsub_rn(b, a), io.m), s_red, io.sum);
    else
        stream_body<float, kVarUnroll>(io.head, io.nvec, f, io.x, io.y, io.m);
}

// Algorithm 1 with the search of Section IV.  The knots and values sit in
// shared memory as (x_j, v_j), padded to 2^L entries with (+inf, v_N),
// 2^L >= N + 1.  The search is unrolled at compile time for that size: L
// steps, each a shared load, a compare and a select (the ternary operator),
// so every query runs the same instructions.  After it, j is the largest
// index with x_j <= x (x clamped to [x_0, x_N]); the interval is i = j + 1,
// or N at x = x_N.  Step 2 divides; step 3 is the two-product lerp (TEX:
// the texture filter at i - 1 + delta + 1/2 instead).  NaN compares false
// everywhere, lands in interval 1 and gives NaN.
template <int L, bool TEX>
struct SearchLerp {
    const float2* s_kv;
    cudaTextureObject_t tex;
    float a, b;
    int N;
    __device__ __forceinline__ float operator()(float x) const
    {
        const float xc = clamp_nan(x, a, b);
        int j = 0;
#pragma unroll
        for (int k = L - 1; k >= 0; --k) {
            const int t = j + (1 << k);
            j = (s_kv[t].x <= xc) ? t : j;
        }
        const int i = min(j + 1, N);
        const float2 l = s_kv[i - 1], r = s_kv[i];
        const float delta = (xc - l.x) / (r.x - l.x);
        if constexpr (TEX) {
            const float yv = tex1D<float>(tex, (float)(i - 1) + delta + 0.5f);
            return xc != xc ? xc : yv;
        } else {
            return (1.0f - delta) * l.y + delta * r.y;
        }
    }
};

template <int L, bool TEX, bool SYNTH>
__global__ void __launch_bounds__(1024) search_kernel(const float* __restrict__ xk_g, const float* __restrict__ vk_g,
                                                      int N, cudaTextureObject_t tex, const StreamIO io)
{
    extern __shared__ float2 s_kv[];
    const float inf = __int_as_float(0x7f800000);
    const float vN = vk_g[N];
    for (int j = threadIdx.x; j < (1 << L); j += blockDim.x)
        s_kv[j] = j <= N ? make_float2(xk_g[j], vk_g[j]) : make_float2(inf, vN);
    __syncthreads();
    const SearchLerp<L, TEX> f{s_kv, tex, s_kv[0].x, s_kv[N].x, N};
    run_variant<SYNTH>(io, f, f.a, f.b, reinterpret_cast<float*>(s_kv));
}

// the largest search depth: 2^14 knot slots of 8 bytes fill 128 KB
constexpr int kMaxSearchLog = 14;

template <bool TEX, bool SYNTH>
struct SearchTable {
    using Kern = void (*)(const float*, const float*, int, cudaTextureObject_t, const StreamIO);
    template <int L>
    static Kern pick(int l)
    {
        if constexpr (L > kMaxSearchLog) {
            return nullptr;
        } else {
            return l == L ? search_kernel<L, TEX, SYNTH> : pick<L + 1>(l);
        }
    }
};

// Mode 1: the interval from the 16-byte (backward-form) index, then the
// texture filter.
struct TexArgs {
    const float4* rec;  // backward records
    const TableHeader* hdr;
    const float* inv_h;
    int K, N, n_smem;
    float a, b, inv_w, off;
};

struct TexLerp {
    const float4* srec;
    const float* s_ih;
    cudaTextureObject_t tex;
    const TexArgs& p;
    int n_stage, max_chain;
    __device__ __forceinline__ float operator()(float x) const
    {
        const float xc = clamp_nan(x, p.a, p.b);
        const int c = cell_of(xc, p.inv_w, p.off, p.K);
        float4 r = (c < n_stage) ? srec[c] : __ldg(p.rec + c);
        for (int g = 0; g < max_chain && xc >= r.x && is_link(r.w); ++g) {
            const int j = link_index(r.w);
            r = (j < n_stage) ? srec[j] : __ldg(p.rec + j);
        }
        const uint32_t jy = __float_as_uint(r.y);
        const bool inside = (jy & kInsideFlag) != 0;  // knot-free cell: 1/h_{j+1} in r.z
        const int j = (int)(jy & ~kInsideFlag);
        float u;  // texel coordinate i - 1 + delta + 1/2
        if (!inside && xc < r.x) {
            u = (float)j + 0.5f - (r.x - xc) * s_ih[j];
        } else if (j < p.N) {
            u = (float)j + 0.5f + (xc - r.x) * (inside ? r.z : s_ih[j + 1]);
        } else {
            u = (float)p.N + 0.5f;
        }
        const float yv = tex1D<float>(tex, u);
        return xc != xc ? xc : yv;
    }
};

template <bool SYNTH>
__global__ void __launch_bounds__(1024) eval_tex_kernel(const TexArgs p, cudaTextureObject_t tex, const StreamIO io)
{
    extern __shared__ float4 s_dyn[];
    float4* srec = s_dyn;                                        // backward-form records
    float* s_ih = reinterpret_cast<float*>(s_dyn + p.n_smem);    // N+2 reciprocal lengths
    const int n_stage = min(p.K + p.hdr->n_chain_b, p.n_smem);
    for (int i = threadIdx.x; i < n_stage; i += blockDim.x) srec[i] = __ldg(p.rec + i);
    for (int i = threadIdx.x; i < p.N + 2; i += blockDim.x) s_ih[i] = p.inv_h[i];
    __syncthreads();
    const TexLerp f{srec, s_ih, tex, p, n_stage, p.hdr->max_chain_b};
    run_variant<SYNTH>(io, f, p.a, p.b, reinterpret_cast<float*>(s_dyn));
}

// Mode 5: a uniform partition needs no search (Section IV): the texture
// coordinate is (x - x_0) N / (x_N - x_0) + 1/2, i.e. i - 1 + delta + 1/2.
struct UniformTex {
    cudaTextureObject_t tex;
    float a, b, scale;  // scale = N / (x_N - x_0)
    __device__ __forceinline__ float operator()(float x) const
    {
        const float xc = clamp_nan(x, a, b);
        const float yv = tex1D<float>(tex, __fmaf_rn(xc - a, scale, 0.5f));
        return xc != xc ? xc : yv;
    }
};

template <bool SYNTH>
__global__ void __launch_bounds__(1024) eval_utex_kernel(const UniformTex f, const StreamIO io)
{
    __shared__ float s_red[32];
    run_variant<SYNTH>(io, f, f.a, f.b, s_red);
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

template <typename IO>
pwl_status launch_eval(pwl_table t, int layout, const IO* x, IO* y, int64_t m, cudaStream_t s)
{
    EvalArgs p{};
    p.recP = t->recP;
    p.recS = t->recS;
    p.recS8 = t->recS8;
    p.xk = t->xk;
    p.rec16 = t->rec16;
    p.hdr = t->hdr;
    p.N = (int)t->N;
    p.a = t->a;
    p.b = t->b;
    size_t smem;
    if (layout == 2) {
        p.K = (int)t->K;
        p.s_staged = 1;
        p.inv_w = t->inv_w;
        p.off = t->off;
        p.w = t->w;
        smem = eval8c_smem_bytes(t);
    } else if (layout == 0) {
        p.K = (int)t->K;
        p.s_staged = forward_side_staged(t->N) ? 1 : 0;
        p.inv_w = t->inv_w;
        p.off = t->off;
        p.w = t->w;
        smem = eval8_smem_bytes(t);
    } else {
        p.K = (int)t->Kb;
        p.n_smem = (int)eval16_smem_records(t);
        p.inv_w = t->inv_w_b;
        p.off = t->off_b;
        smem = eval16_smem_bytes(t);
        if (p.n_smem < p.K) return fail(PWL_ENOTSUP, "16-byte index of %d cells does not fit one CTA", p.K);
    }
    stream_split<IO>(x, y, m, &p.head, &p.nvec);
    const DeviceInfo& di = device_info();
    if (smem > di.smem_optin) return fail(PWL_ENOTSUP, "forward index of %zu bytes does not fit one CTA", smem);
    const bool two = di.smem_per_sm >= 2 * (smem + 1024);
    void (*kern)(const EvalArgs, const IO*, IO*, int64_t);
    if (layout == 0)
        kern = two ? eval_kernel<IO, 0, 2> : eval_kernel<IO, 0, 1>;
    else if (layout == 2)
        kern = two ? eval_kernel<IO, 2, 2> : eval_kernel<IO, 2, 1>;
    else
        kern = two ? eval_kernel<IO, 1, 2> : eval_kernel<IO, 1, 1>;
    int max_grid = 0;
    PWL_CUDA_TRY(occupancy_grid(kern, 1024, smem, &max_grid));
    // small launches: no more CTAs than there are unrolled vector groups,
    // but one per SM while each gets a few vectors per warp (the CTAs stage
    // the index concurrently, so spreading costs no latency and uses every
    // SM's loads); tiny ones do not stage the index in idle CTAs
    const int grid = stream_grid(max_grid, p.nvec + (m - p.nvec * Vec<IO>::n), 1024, kUnroll);
    kern<<<grid, 1024, smem, s>>>(p, x, y, m);
    PWL_CHECK_LAUNCH("eval_kernel");
    return PWL_OK;
}

pwl_status launch_synth(pwl_table t, int layout, uint32_t seed, int64_t m, double* sum, cudaStream_t s)
{
    EvalArgs p{};
    p.recP = t->recP;
    p.recS = t->recS;
    p.recS8 = t->recS8;
    p.xk = t->xk;
    p.rec16 = t->rec16;
    p.hdr = t->hdr;
    p.N = (int)t->N;
    p.a = t->a;
    p.b = t->b;
    size_t smem;
    if (layout == 2) {
        p.K = (int)t->K;
        p.s_staged = 1;
        p.inv_w = t->inv_w;
        p.off = t->off;
        p.w = t->w;
        smem = eval8c_smem_bytes(t);
    } else if (layout == 0) {
        p.K = (int)t->K;
        p.s_staged = forward_side_staged(t->N) ? 1 : 0;
        p.inv_w = t->inv_w;
        p.off = t->off;
        p.w = t->w;
        smem = eval8_smem_bytes(t);
    } else {
        p.K = (int)t->Kb;
        p.n_smem = (int)eval16_smem_records(t);
        p.inv_w = t->inv_w_b;
        p.off = t->off_b;
        smem = eval16_smem_bytes(t);
        if (p.n_smem < p.K) return fail(PWL_ENOTSUP, "16-byte index of %d cells does not fit one CTA", p.K);
    }
    const DeviceInfo& di = device_info();
    if (smem > di.smem_optin) return fail(PWL_ENOTSUP, "forward index of %zu bytes does not fit one CTA", smem);
    const bool two = di.smem_per_sm >= 2 * (smem + 1024);
    void (*kern)(const EvalArgs, uint32_t, int64_t, double*);
    if (layout == 0)
        kern = two ? eval_synth_kernel<0, 2> : eval_synth_kernel<0, 1>;
    else if (layout == 2)
        kern = two ? eval_synth_kernel<2, 2> : eval_synth_kernel<2, 1>;
    else
        kern = two ? eval_synth_kernel<1, 2> : eval_synth_kernel<1, 1>;
    int max_grid = 0;
    PWL_CUDA_TRY(occupancy_grid(kern, 1024, smem, &max_grid));
    const int grid = (int)std::min<int64_t>(max_grid, std::max<int64_t>(1, (m + 4095) / 4096));
    kern<<<grid, 1024, smem, s>>>(p, seed, m, sum);
    PWL_CHECK_LAUNCH("eval_synth_kernel");
    return PWL_OK;
}

// The texels are the table's rounded values (FP32, or FP16 for FP16
// tables), copied on the caller's stream after the kernels that wrote them.
pwl_status copy_texels(pwl_table t, cudaStream_t s)
{
    const bool half_texels = (t->dtype == PWL_FP16);
    const void* src = half_texels ? t->vstore : (const void*)t->vk;
    const size_t row = (half_texels ? 2 : 4) * (size_t)(t->N + 1);
    PWL_CUDA_TRY(cudaMemcpy2DToArrayAsync(t->tex_array, 0, 0, src, row, row, 1, cudaMemcpyDeviceToDevice, s));
    return PWL_OK;
}

pwl_status ensure_texture(pwl_table t, cudaStream_t s)
{
    if (t->tex) return PWL_OK;
    int maxa = 0;
    cudaDeviceGetAttribute(&maxa, cudaDevAttrMaxTexture1DWidth, t->device);
    if (t->N + 1 > maxa)
        return fail(PWL_ENOTSUP, "texture path supports at most %d knots", maxa);
    const bool half_texels = (t->dtype == PWL_FP16);
    cudaChannelFormatDesc cd = half_texels ? cudaCreateChannelDescHalf() : cudaCreateChannelDesc<float>();
    PWL_CUDA_TRY(dev_malloc_array(&t->tex_array, &cd, (size_t)t->N + 1));
    // from here on a failure frees the array, so that a later call starts afresh
    auto undo = [&](pwl_status st) {
        cudaFreeArray(t->tex_array);
        t->tex_array = nullptr;
        return st;
    };
    pwl_status st = copy_texels(t, s);
    if (st != PWL_OK) return undo(st);
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = t->tex_array;
    cudaTextureDesc td{};
    td.addressMode[0] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModeLinear;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    cudaError_t e = cudaCreateTextureObject(&t->tex, &rd, &td, nullptr);
    if (e != cudaSuccess) {
        t->tex = 0;
        return undo(cuda_fail(e, "cudaCreateTextureObject"));
    }
    return PWL_OK;
}

}  // namespace

pwl_status refresh_texture(pwl_table t, cudaStream_t s)
{
    return t->tex ? copy_texels(t, s) : PWL_OK;
}

namespace {

// Modes 0, 1, 4 and 5 on a query stream (synth = false: io.x, io.y, io.m)
// or on generated queries (synth = true: io.seed, io.m, io.sum).
pwl_status launch_variant(pwl_table t, int mode, bool synth, StreamIO io, cudaStream_t s)
{
    const DeviceInfo& di = device_info();
    if (!synth) stream_split<float>(io.x, io.y, io.m, &io.head, &io.nvec);
    const int64_t units = synth ? (io.m + 3) / 4 : io.nvec + (io.m - io.nvec * 4);
    if (mode == 1 || mode == 4 || mode == 5) {
        pwl_status st = ensure_texture(t, s);
        if (st != PWL_OK) return st;
    }
    int max_grid = 0;
    if (mode == 0 || mode == 4) {
        int L = 1;
        while (((int64_t)1 << L) < t->N + 1) ++L;
        if (L > kMaxSearchLog)
            return fail(PWL_ENOTSUP, "search path stages at most 2^%d knots (N = %lld)", kMaxSearchLog,
                        (long long)t->N);
        void (*kern)(const float*, const float*, int, cudaTextureObject_t, const StreamIO);
        if (mode == 0)
            kern = synth ? SearchTable<false, true>::pick<1>(L) : SearchTable<false, false>::pick<1>(L);
        else
            kern = synth ? SearchTable<true, true>::pick<1>(L) : SearchTable<true, false>::pick<1>(L);
        const size_t smem = std::max<size_t>(sizeof(float2) << L, 128);
        PWL_CUDA_TRY(occupancy_grid(kern, 1024, smem, &max_grid));
        kern<<<stream_grid(max_grid, units, 1024, kVarUnroll), 1024, smem, s>>>(t->xk, t->vk, (int)t->N, t->tex, io);
        PWL_CHECK_LAUNCH("search_kernel");
        return PWL_OK;
    }
    if (mode == 5) {
        void (*kern)(const UniformTex, const StreamIO) = synth ? eval_utex_kernel<true> : eval_utex_kernel<false>;
        const UniformTex f{t->tex, t->a, t->b, (float)((double)t->N / ((double)t->b - (double)t->a))};
        PWL_CUDA_TRY(occupancy_grid(kern, 1024, 0, &max_grid));
        kern<<<stream_grid(max_grid, units, 1024, kVarUnroll), 1024, 0, s>>>(f, io);
        PWL_CHECK_LAUNCH("eval_utex_kernel");
        return PWL_OK;
    }
    // mode 1
    const size_t fixed = sizeof(float) * (size_t)(t->N + 2);
    if (fixed + 1024 > di.smem_optin) return fail(PWL_ENOTSUP, "table too large for the texture path");
    TexArgs p{};
    p.rec = t->rec_b;
    p.hdr = t->hdr;
    p.inv_h = t->inv_h;
    p.K = (int)t->Kb;
    p.N = (int)t->N;
    p.n_smem = (int)std::min<int64_t>(t->Kb + t->chain_reserve_b, (int64_t)((di.smem_optin - fixed) / 16));
    p.a = t->a;
    p.b = t->b;
    p.inv_w = t->inv_w_b;
    p.off = t->off_b;
    const size_t smem = std::max<size_t>(16 * (size_t)p.n_smem + fixed, 128);
    void (*kern)(const TexArgs, cudaTextureObject_t, const StreamIO) =
        synth ? eval_tex_kernel<true> : eval_tex_kernel<false>;
    PWL_CUDA_TRY(occupancy_grid(kern, 1024, smem, &max_grid));
    kern<<<stream_grid(max_grid, units, 1024, kVarUnroll), 1024, smem, s>>>(p, t->tex, io);
    PWL_CHECK_LAUNCH("eval_tex_kernel");
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
        return launch_eval<float>(t, t->layout, static_cast<const float*>(d_x), static_cast<float*>(d_y), m, s);
    case PWL_BF16:
        return launch_eval<__nv_bfloat16>(t, t->layout, static_cast<const __nv_bfloat16*>(d_x),
                                          static_cast<__nv_bfloat16*>(d_y), m, s);
    case PWL_FP16:
        return launch_eval<__half>(t, t->layout, static_cast<const __half*>(d_x), static_cast<__half*>(d_y), m, s);
    }
    return fail(PWL_EINVAL, "unknown io dtype %d", io_dtype);
}

pwl_status pwl_eval_synthetic(pwl_table t, uint32_t seed, int64_t m, double* d_sum, void* stream)
{
    clear_error();
    if (!t) return fail(PWL_EINVAL, "table is NULL");
    if (m < 0 || m > ((int64_t)1 << 32)) return fail(PWL_EINVAL, "m must be in [0, 2^32]");
    if (!d_sum) return fail(PWL_EINVAL, "d_sum is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return fail(PWL_EINVAL, "table lives on device %d, current device is %d", t->device, dev);
    if (m == 0) return PWL_OK;
    return launch_synth(t, t->layout, seed, m, d_sum, as_stream(stream));
}

pwl_status pwl_eval_synthetic_variant(pwl_table t, int32_t mode, uint32_t seed, int64_t m, double* d_sum,
                                      void* stream)
{
    clear_error();
    if (!t) return fail(PWL_EINVAL, "table is NULL");
    if (mode < 0 || mode > 6) return fail(PWL_EINVAL, "unknown mode %d", mode);
    if (m < 0 || m > ((int64_t)1 << 32)) return fail(PWL_EINVAL, "m must be in [0, 2^32]");
    if (!d_sum) return fail(PWL_EINVAL, "d_sum is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return fail(PWL_EINVAL, "table lives on device %d, current device is %d", t->device, dev);
    if (m == 0) return PWL_OK;
    if (mode == 2 || mode == 3) return launch_synth(t, mode - 2, seed, m, d_sum, as_stream(stream));
    if (mode == 6) return launch_synth(t, 2, seed, m, d_sum, as_stream(stream));
    StreamIO io{};
    io.m = m;
    io.seed = seed;
    io.sum = d_sum;
    return launch_variant(t, mode, true, io, as_stream(stream));
}

pwl_status pwl_eval_variant(pwl_table t, int32_t mode, const float* d_x, float* d_y, int64_t m,
                            void* stream)
{
    clear_error();
    pwl_status st = check_common(t, d_x, d_y, m);
    if (st != PWL_OK) return st;
    if (mode < 0 || mode > 6) return fail(PWL_EINVAL, "unknown mode %d", mode);
    if (m == 0) return PWL_OK;
    cudaStream_t s = as_stream(stream);
    if (mode == 2 || mode == 3) return launch_eval<float>(t, mode - 2, d_x, d_y, m, s);
    if (mode == 6) return launch_eval<float>(t, 2, d_x, d_y, m, s);
    StreamIO io{};
    io.x = d_x;
    io.y = d_y;
    io.m = m;
    return launch_variant(t, mode, false, io, s);
}

}  // extern "C"
