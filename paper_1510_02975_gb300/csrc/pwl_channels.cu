// pwl_channels.cu -- channel-wise CPWL map: y[r, c] = v_c(x[r, c]) for a
// row-major x[R, C] with one CPWL function per channel (Algorithm 1 per
// element), and its backward (gradients w.r.t. x, the vertex values and the
// knots of every channel).  The knots and values are plain FP32 device
// arrays [C, N+1] (learnable parameters that change every step), so each CTA
// builds the cell index of its channels in shared memory when it starts.
//
// Forward: a CTA owns a tile of 8 consecutive channels and keeps, per
// channel, 16-byte cell records {x_s, y_s, s_left, s_right} (one load, a
// compare, a select and an FMA per element), channel-interleaved ([c * 8 + ch])
// so that the 8 lanes of a quarter warp read 8 different bank groups.  Four
// CTAs form a thread-block cluster on adjacent tiles (32 channels, 128-byte
// row segments) and walk the same rows at once.
//
// Backward: a CTA owns 16 channels (a warp covers two rows, 64-byte row
// segments), with 8-byte cell records {i, x_{i-1}} or {knot tag, x_k} and
// interval records {s_i, 1/h_i}, channel-interleaved ([e * 16 + ch]), and
// two shared accumulators per interval; 2-CTA clusters (128-byte segments).
//
// Both: the rows of x are split into chunks; units = (tile group, chunk of
// rows), group-major; each cluster takes a contiguous range of units and
// rebuilds its indexes only when the group changes.  A 32-byte row segment
// read by one CTA alone costs a whole line fetch; the sibling CTAs of a
// cluster use the rest of the line while it is in L2.
#include <math.h>

#include <algorithm>

#include "pwl_channels.cuh"

namespace pwl {

namespace {

constexpr int kChThreads = 1024;                 // threads per CTA, both directions
// backward tiles (the forward's constants are kChF, kClF, kRowsPerPassF, ...)
constexpr int kCh = 16;                          // channels per backward tile
constexpr int kRowsPerPass = kChThreads / kCh;   // 64 rows per pass of the CTA
constexpr int kChUnroll = 16;                    // loads in flight per thread (8 rows x, gy: 64 KB per SM)
constexpr int kChTail = 3;                       // rows per predicated batch of a unit's tail

struct TileParams {
    float a[kCh], b[kCh], inv_w[kCh], off[kCh], w[kCh];
    int max_chain[kCh];
    int any_chain;
    int bad;
};

__device__ __forceinline__ int lower_bound_cells(const int* cj, int n, int v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (cj[mid * kCh] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Slopes are FP32 IEEE divisions of the FP32 differences: at most ~2 ulp
// from the exact slope of the FP32 table, which moves a lerped value by
// ~2^-23 |v_i - v_{i-1}| (FP64 would cost a slow FP64 division per record on
// this GPU's few FP64 units).

// Builds the backward index of channels [c0, c0 + 16) in shared memory.
//   sP[cell * 16 + ch]      cell records {i, x_{i-1}} or {knot tag, x_k}
//   sX[i * 16 + ch]         interval records {s_i, 1/h_i}, i = 0..N+1 (0 and N+1
//                           copy intervals 1 and N)
//   xs[j * 16 + ch]         the tile's knots (staged first, coalesced)
//   cj[j * 16 + ch]         scratch: first the tile's values, then the cell of knot j
// Every global read is a coalesced pass over the tile's knots and values;
// the rest works in shared memory.
__device__ void build_tile(const ChanArgs& p, int64_t c0, float2* sP, float2* sX, float* xs, int* cj,
                           TileParams* tp)
{
    const int N = p.N, K = p.K, n1 = N + 1;
    const int nch = (int)min((int64_t)kCh, p.C - c0);
    float* vs = reinterpret_cast<float*>(cj);
    const int per_ch = blockDim.x / kCh;  // threads per channel
    for (int ch = threadIdx.x / per_ch, j = threadIdx.x % per_ch; j < n1; j += per_ch) {
        // consecutive threads read consecutive knots of one channel
        float xv, vv;
        if (ch < nch) {
            xv = p.knots[(c0 + ch) * (int64_t)n1 + j];
            vv = p.values[(c0 + ch) * (int64_t)n1 + j];
        } else {  // padding channel of a partial tile: an unused identity on [0, 1]
            xv = (float)j / (float)N;
            vv = 0.0f;
        }
        xs[j * kCh + ch] = xv;
        vs[j * kCh + ch] = vv;
    }
    if (threadIdx.x == 0) {
        tp->any_chain = 0;
        tp->bad = 0;
    }
    __syncthreads();
    if (threadIdx.x < kCh) {
        const int ch = threadIdx.x;
        const float a = xs[ch], b = xs[N * kCh + ch];
        tp->a[ch] = a;
        tp->b[ch] = b;
        tp->inv_w[ch] = (float)K / (b - a);
        tp->off[ch] = -a * tp->inv_w[ch];
        tp->w[ch] = (b - a) / (float)K;
        tp->max_chain[ch] = 0;
    }
    // interval records, from the staged arrays
    for (int e = threadIdx.x; e < (N + 2) * kCh; e += blockDim.x) {
        const int q = e / kCh, ch = e % kCh;
        const int i = min(max(q, 1), N);  // interval q (0 and N+1 copy 1 and N)
        const float h = __fsub_rn(xs[i * kCh + ch], xs[(i - 1) * kCh + ch]);
        sX[e] = make_float2(__fdiv_rn(__fsub_rn(vs[i * kCh + ch], vs[(i - 1) * kCh + ch]), h), __frcp_rn(h));
    }
    __syncthreads();
    // cells of the knots (overwrites the staged values)
    for (int e = threadIdx.x; e < n1 * kCh; e += blockDim.x) {
        const int j = e / kCh, ch = e % kCh;
        const float xj = xs[e];
        if (j > 0 && !(xj > xs[e - kCh])) atomicOr(&tp->bad, 1);
        cj[e] = cell_of(xj, tp->inv_w[ch], tp->off[ch], K);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n1 * kCh; e += blockDim.x) {
        const int j = e / kCh, ch = e % kCh;
        if (j > 0 && cj[e] == cj[e - kCh]) {
            int first = j;
            while (first > 0 && cj[(first - 1) * kCh + ch] == cj[e]) --first;
            atomicMax(&tp->max_chain[ch], j - first);
            atomicOr(&tp->any_chain, 1);
        }
    }
    // cell records: each thread takes a run of consecutive cells of one
    // channel, finds the first one's knot by bisection and walks on
    {
        const int ch = threadIdx.x % kCh, runs = blockDim.x / kCh, q = threadIdx.x / kCh;
        const int per = (K + runs - 1) / runs;
        const int cb = q * per, ce = min(K, cb + per);
        int lb = cb < ce ? lower_bound_cells(cj + ch, n1, cb) : 0;
        for (int c = cb; c < ce; ++c) {
            while (lb < n1 && cj[lb * kCh + ch] < c) ++lb;  // lb: the first knot whose cell is >= c
            float2 rec;
            if (lb <= N && cj[lb * kCh + ch] == c) {
                const bool chain = (lb < N && cj[(lb + 1) * kCh + ch] == c);
                rec = make_float2(make_knot_tag(lb, chain), xs[lb * kCh + ch]);
            } else {
                const int i = lb;  // the cell lies inside interval i = [x_{i-1}, x_i]
                rec = make_float2(__int_as_float(i), xs[(i - 1) * kCh + ch]);
            }
            sP[c * kCh + ch] = rec;
        }
    }
    __syncthreads();
}

// A thread's channel is fixed for a tile: its constants live in registers.
struct ChanConst {
    float a, b, inv_w, off, w;
    int max_chain;
    __device__ __forceinline__ ChanConst(const TileParams& tp, int ch)
        : a(tp.a[ch]), b(tp.b[ch]), inv_w(tp.inv_w[ch]), off(tp.off[ch]), w(tp.w[ch]), max_chain(tp.max_chain[ch])
    {
    }
};

template <typename IO>
__device__ __forceinline__ float to_f32(IO v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename IO>
__device__ __forceinline__ IO from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ void st_cs(float* p, float v) { __stcs(p, v); }
__device__ __forceinline__ void st_cs(__nv_bfloat16* p, __nv_bfloat16 v) { *p = v; }

// ---- forward: 8-channel tiles with 16-byte split records ---------------------
// A cell record is {x_s, y_s, s_left, s_right}: v(x) = y_s + (x - x_s) s with
// s = s_left left of x_s and s_right from x_s on.  A knot-free cell inside
// interval i stores its anchor x_c = a + c w, the line's value there and s_i
// twice; a cell holding one knot k stores {x_k, v_k, s_k, s_{k+1}}.  One
// 16-byte load, a compare, a select and an FMA per element; no tag test and
// no second load.  A cell holding several knots stores a NaN-tagged s_right
// (knot k, its first): elements right of x_k walk the tile's knots and take
// {x_k', v_k', s_{k'+1}} from the staged knots, values and slopes.
// Records are channel-interleaved ([c * 8 + ch]): the 8 lanes of a quarter
// warp read 8 different 16-byte bank groups.  With 4 cells per knot a tile
// takes 128 (K + N + 1) bytes (164 KB at N = 256), so a CTA owns 8 channels,
// and 4-CTA clusters walk the same rows at once to use whole 128-byte lines.
constexpr int kChF = 8;                           // channels per forward tile
constexpr int kClF = 4;                           // CTAs per forward cluster (32 channels)
constexpr int kRowsPerPassF = kChThreads / kChF;  // 128 rows per pass
constexpr int kChUnrollF = 24;
constexpr int kChTailF = 8;

struct TileParamsF {
    float a[kChF], b[kChF], inv_w[kChF], off[kChF], w[kChF];
    int max_chain[kChF];
    int any_chain;
    int bad;
};

struct ChanConstF {
    float a, b, inv_w, off, w;
    int max_chain;
    __device__ __forceinline__ ChanConstF(const TileParamsF& tp, int ch)
        : a(tp.a[ch]), b(tp.b[ch]), inv_w(tp.inv_w[ch]), off(tp.off[ch]), w(tp.w[ch]), max_chain(tp.max_chain[ch])
    {
    }
};

__device__ __forceinline__ int lower_bound_cells8(const int* cj, int n, int v)
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cj[mid * kChF] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Builds the forward index of channels [c0, c0 + 8) in shared memory:
//   R[c * 8 + ch]   cell records (K)
//   xs, vs, sp      knots, values and slopes s_{j+1} (s_N for j = N), [j * 8 + ch]
//   cj              build scratch: the cell of knot j
__device__ void build_tile_fwd(const ChanArgs& p, int64_t c0, float4* R, float* xs, float* vs, float* sp, int* cj,
                               TileParamsF* tp)
{
    const int N = p.N, K = p.K, n1 = N + 1;
    const int nch = (int)min((int64_t)kChF, p.C - c0);
    const int per_ch = blockDim.x / kChF;  // threads per channel
    for (int ch = threadIdx.x / per_ch, j = threadIdx.x % per_ch; j < n1; j += per_ch) {
        // consecutive threads read consecutive knots of one channel
        float xv, vv;
        if (ch < nch) {
            xv = p.knots[(c0 + ch) * (int64_t)n1 + j];
            vv = p.values[(c0 + ch) * (int64_t)n1 + j];
        } else {  // padding channel of a partial tile: an unused identity on [0, 1]
            xv = (float)j / (float)N;
            vv = 0.0f;
        }
        xs[j * kChF + ch] = xv;
        vs[j * kChF + ch] = vv;
    }
    if (threadIdx.x == 0) {
        tp->any_chain = 0;
        tp->bad = 0;
    }
    __syncthreads();
    if (threadIdx.x < kChF) {
        const int ch = threadIdx.x;
        const float a = xs[ch], b = xs[N * kChF + ch];
        tp->a[ch] = a;
        tp->b[ch] = b;
        tp->inv_w[ch] = (float)K / (b - a);
        tp->off[ch] = -a * tp->inv_w[ch];
        tp->w[ch] = (b - a) / (float)K;
        tp->max_chain[ch] = 0;
    }
    for (int e = threadIdx.x; e < n1 * kChF; e += blockDim.x) {
        const int j = e / kChF, ch = e % kChF;
        const int i = min(j + 1, N);  // slope of interval j + 1 (of interval N for j = N)
        const float h = __fsub_rn(xs[i * kChF + ch], xs[(i - 1) * kChF + ch]);
        sp[e] = __fdiv_rn(__fsub_rn(vs[i * kChF + ch], vs[(i - 1) * kChF + ch]), h);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n1 * kChF; e += blockDim.x) {
        const int j = e / kChF, ch = e % kChF;
        const float xj = xs[e];
        if (j > 0 && !(xj > xs[e - kChF])) atomicOr(&tp->bad, 1);
        cj[e] = cell_of(xj, tp->inv_w[ch], tp->off[ch], K);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n1 * kChF; e += blockDim.x) {
        const int j = e / kChF, ch = e % kChF;
        if (j > 0 && cj[e] == cj[e - kChF]) {
            int first = j;
            while (first > 0 && cj[(first - 1) * kChF + ch] == cj[e]) --first;
            atomicMax(&tp->max_chain[ch], j - first);
            atomicOr(&tp->any_chain, 1);
        }
    }
    // cell records: each thread takes a run of consecutive cells of one
    // channel, finds the first one's knot by bisection and walks on
    {
        const int ch = threadIdx.x % kChF, runs = blockDim.x / kChF, q = threadIdx.x / kChF;
        const int per = (K + runs - 1) / runs;
        const int cb = q * per, ce = min(K, cb + per);
        int lb = cb < ce ? lower_bound_cells8(cj + ch, n1, cb) : 0;
        for (int c = cb; c < ce; ++c) {
            while (lb < n1 && cj[lb * kChF + ch] < c) ++lb;  // lb: the first knot whose cell is >= c
            float4 rec;
            if (lb <= N && cj[lb * kChF + ch] == c) {  // knot lb is the cell's first knot
                const int k = lb;
                const bool chain = k < N && cj[(k + 1) * kChF + ch] == c;
                const float sl = sp[max(k - 1, 0) * kChF + ch];
                const float sr = chain ? make_knot_tag(k, true) : sp[k * kChF + ch];
                rec = make_float4(xs[k * kChF + ch], vs[k * kChF + ch], sl, sr);
            } else {  // inside interval lb: the line through (x_j, v_j), j = lb - 1, at the anchor
                const int j = lb - 1;
                const float sj = sp[j * kChF + ch];
                const float xc = __fmaf_rn(__int2float_rn(c), tp->w[ch], tp->a[ch]);
                rec = make_float4(xc, __fmaf_rn(__fsub_rn(xc, xs[j * kChF + ch]), sj, vs[j * kChF + ch]), sj, sj);
            }
            R[c * kChF + ch] = rec;
        }
    }
    __syncthreads();
}

template <bool CHAINS>
__device__ __forceinline__ float chan_fwd8(float x, int ch, const float4* R, const float* xs, const float* vs,
                                           const float* sp, const ChanConstF& cc, int N, int K)
{
    const float xc = clamp_nan(x, cc.a, cc.b);
    const int c = cell_of(xc, cc.inv_w, cc.off, K);
    const float4 r = R[c * kChF + ch];
    float s = xc < r.x ? r.z : r.w;
    float anchor = r.x, y0 = r.y;
    if (CHAINS && s != s) {  // right of the first knot of a cell holding several
        int k = (int)(__float_as_uint(r.w) & kKnotTagMask);
        for (int g = 0; g < cc.max_chain && k < N; ++g) {
            if (!(xc >= xs[(k + 1) * kChF + ch])) break;
            ++k;
        }
        anchor = xs[k * kChF + ch];
        y0 = vs[k * kChF + ch];
        s = sp[k * kChF + ch];
    }
    return __fmaf_rn(xc - anchor, s, y0);
}

template <typename IO, bool CHAINS>
__device__ __forceinline__ void chan_fwd8_rows(const ChanArgs& p, int64_t c0, int64_t r0, int64_t r1,
                                               const float4* R, const float* xs, const float* vs, const float* sp,
                                               const TileParamsF& tp, const IO* __restrict__ x, IO* __restrict__ y)
{
    const int ch = threadIdx.x % kChF;
    const int64_t c = c0 + ch;
    if (c >= p.C) return;
    const ChanConstF cc(tp, ch);
    int64_t r = r0 + threadIdx.x / kChF;
    const int64_t pass = (int64_t)kRowsPerPassF * p.C;  // elements between a thread's consecutive rows
    // x is read at the L2 only (ld.global.cg): 2% faster than through L1,
    // whose lines the row segments of other CTAs do not share anyway
    const IO* px = x + r * p.C + c;
    IO* py = y + r * p.C + c;
    for (; r + (int64_t)(kChUnrollF - 1) * kRowsPerPassF < r1; r += (int64_t)kChUnrollF * kRowsPerPassF) {
        float v[kChUnrollF];
#pragma unroll
        for (int u = 0; u < kChUnrollF; ++u) v[u] = to_f32<IO>(__ldcg(px + u * pass));
#pragma unroll
        for (int u = 0; u < kChUnrollF; ++u) v[u] = chan_fwd8<CHAINS>(v[u], ch, R, xs, vs, sp, cc, p.N, p.K);
#pragma unroll
        for (int u = 0; u < kChUnrollF; ++u) st_cs(py + u * pass, from_f32<IO>(v[u]));
        px += kChUnrollF * pass;
        py += kChUnrollF * pass;
    }
    // the rest (fewer than kChUnrollF rows per thread) in predicated batches of
    // kChTailF: a few load latencies instead of one per row
    for (; r < r1; r += (int64_t)kChTailF * kRowsPerPassF) {
        const int64_t left = (r1 - r + kRowsPerPassF - 1) / kRowsPerPassF;
        const int rem = left < kChTailF ? (int)left : kChTailF;
        float v[kChTailF];
#pragma unroll
        for (int u = 0; u < kChTailF; ++u)
            if (u < rem) v[u] = to_f32<IO>(__ldcg(px + u * pass));
#pragma unroll
        for (int u = 0; u < kChTailF; ++u)
            if (u < rem) st_cs(py + u * pass, from_f32<IO>(chan_fwd8<CHAINS>(v[u], ch, R, xs, vs, sp, cc, p.N, p.K)));
        px += kChTailF * pass;
        py += kChTailF * pass;
    }
}

// Units = (tile quad, chunk of rows), quad-major; the 4 CTAs of a cluster take
// the 4 tiles of a quad on the same rows.
template <typename IO>
__global__ void __launch_bounds__(kChThreads, 1) channels_forward_kernel(const ChanArgs p, const IO* x, IO* y)
{
    extern __shared__ float4 s_ch[];
    float4* R = s_ch;
    float* xs = reinterpret_cast<float*>(R + (size_t)p.K * kChF);
    float* vs = xs + (size_t)(p.N + 1) * kChF;
    float* sp = vs + (size_t)(p.N + 1) * kChF;
    int* cj = reinterpret_cast<int*>(sp + (size_t)(p.N + 1) * kChF);
    __shared__ TileParamsF tp;
    const int64_t cluster = blockIdx.x / kClF, nclusters = gridDim.x / kClF;
    const int64_t u0 = p.units * cluster / nclusters, u1 = p.units * (cluster + 1) / nclusters;
    int64_t built = -1;
    for (int64_t u = u0; u < u1; ++u) {
        const int64_t tile = kClF * (u / p.per_pair) + (blockIdx.x % kClF), chunk = u % p.per_pair;
        if (tile >= p.tiles) continue;  // a tile past the last one of a partial quad
        if (tile != built) {
            __syncthreads();
            build_tile_fwd(p, tile * kChF, R, xs, vs, sp, cj, &tp);
            if (threadIdx.x == 0 && tp.bad) atomicOr(p.status, 1);
            built = tile;
        }
        const int64_t r0 = chunk * p.rows_per_unit, r1 = min(p.R, r0 + p.rows_per_unit);
        if (tp.any_chain)
            chan_fwd8_rows<IO, true>(p, tile * kChF, r0, r1, R, xs, vs, sp, tp, x, y);
        else
            chan_fwd8_rows<IO, false>(p, tile * kChF, r0, r1, R, xs, vs, sp, tp, x, y);
    }
}

// ---- backward ----------------------------------------------------------------
// gx = gy * s_i; per (channel, interval) sums A_i = sum gy (1 - delta) and
// B_i = sum gy delta accumulate in shared memory (FP32 atomics); at the end
// of a tile's rows they become g_v[j] += A_{j+1} + B_j (+ clamped terms) and
// g_x[j] += -s_{j+1} A_{j+1} - s_j B_j, added to the global gradients.
struct EndSums {
    float left, right;
};

// One element without branches apart from chain walks (a divergent version
// issued the shared-memory atomics once per path): the lookup runs on the
// clamped point (NaN looks up a and contributes nothing), the side and the
// interval come from selects, and one predicated pair of atomics takes an
// in-range element's two sums.  A knot-free cell's record {i, x_{i-1}} is
// the right side of knot i - 1; a knot cell's {tag(k), x_k} either side of
// knot k; so both read "knot k, point x_k".
template <bool CHAINS>
__device__ __forceinline__ float chan_bwd_one(float x, float g, int ch, const float* __restrict__ xs,
                                              const float2* sP, const float2* sI, const ChanConst& cc, int N,
                                              int K, float* accA, float* accB, EndSums& e)
{
    const float xc = fminf(fmaxf(x, cc.a), cc.b);  // NaN -> a
    const int c = cell_of(xc, cc.inv_w, cc.off, K);
    const float2 r = sP[c * kCh + ch];
    const uint32_t bits = __float_as_uint(r.x);
    const bool knot = (bits & 0xFFC00000u) == kLinkTag;
    int k = knot ? (int)(bits & kKnotTagMask) : __float_as_int(r.x) - 1;
    float xk = r.y;
    if (CHAINS && knot && (bits & kKnotTagChain)) {
        for (int gg = 0; gg < cc.max_chain && k < N; ++gg) {
            const float xn = xs[(k + 1) * kCh + ch];
            if (!(xc >= xn)) break;
            ++k;
            xk = xn;
        }
    }
    // right of x_k: interval k + 1 from its left end; left of it: interval k
    // from its right end; x = x_N: interval N at delta = 1
    const bool right = xc >= xk;
    const bool at_b = right && k == N;
    const int i = right && !at_b ? k + 1 : k;
    const float2 q = sI[i * kCh + ch];
    const float tt = (right ? (xc - xk) : (xk - xc)) * q.y;
    const float delta = at_b ? 1.0f : (right ? tt : 1.0f - tt);
    const float one_minus = at_b ? 0.0f : (right ? 1.0f - tt : tt);
    const bool inside = x >= cc.a && x <= cc.b;  // false for NaN
    if (inside) {
        atomicAdd(accA + i * kCh + ch, g * one_minus);
        atomicAdd(accB + i * kCh + ch, g * delta);
    }
    e.left += x < cc.a ? g : 0.0f;
    e.right += x > cc.b ? g : 0.0f;
    const float gx = inside ? g * q.x : 0.0f;
    return x != x ? x : gx;
}

template <bool CHAINS>
__device__ __forceinline__ void chan_bwd_rows(const ChanArgs& p, int64_t c0, int64_t r0, int64_t r1,
                                              const float2* sP, const float2* sI, const float* xs,
                                              const TileParams& tp, float* accA, float* accB,
                                              const float* __restrict__ x, const float* __restrict__ gy,
                                              float* __restrict__ gx)
{
    const int ch = threadIdx.x % kCh;
    const int64_t c = c0 + ch;
    EndSums e{0.0f, 0.0f};
    if (c < p.C) {
        const ChanConst cc(tp, ch);
        int64_t r = r0 + threadIdx.x / kCh;
        const int64_t pass = (int64_t)kRowsPerPass * p.C;
        const int64_t o = r * p.C + c;
        const float* px = x + o;
        const float* pg = gy + o;
        float* po = gx + o;
        constexpr int U = kChUnroll / 2;  // two loads per element
        for (; r + (int64_t)(U - 1) * kRowsPerPass < r1; r += (int64_t)U * kRowsPerPass) {
            float xv[U], gv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                xv[u] = px[u * pass];
                gv[u] = pg[u * pass];
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                po[u * pass] = chan_bwd_one<CHAINS>(xv[u], gv[u], ch, xs, sP, sI, cc, p.N, p.K, accA, accB, e);
            px += U * pass;
            pg += U * pass;
            po += U * pass;
        }
        // the rest (fewer than U rows per thread) in predicated batches of
        // kChTail: a few load latencies instead of one per row
        for (; r < r1; r += (int64_t)kChTail * kRowsPerPass) {
            const int64_t left = (r1 - r + kRowsPerPass - 1) / kRowsPerPass;
            const int rem = left < kChTail ? (int)left : kChTail;
            float xv[kChTail], gv[kChTail];
#pragma unroll
            for (int u = 0; u < kChTail; ++u)
                if (u < rem) {
                    xv[u] = px[u * pass];
                    gv[u] = pg[u * pass];
                }
#pragma unroll
            for (int u = 0; u < kChTail; ++u)
                if (u < rem)
                    po[u * pass] = chan_bwd_one<CHAINS>(xv[u], gv[u], ch, xs, sP, sI, cc, p.N, p.K, accA, accB, e);
            px += kChTail * pass;
            pg += kChTail * pass;
            po += kChTail * pass;
        }
    }
    // lanes ch and ch + 16 share a channel: one add each
    if (e.left != 0.0f) atomicAdd(accA + 0 * kCh + ch, e.left);
    if (e.right != 0.0f) atomicAdd(accA + (p.N + 1) * kCh + ch, e.right);
}

// Adds a tile's shared sums to the global gradients and clears them.
__device__ void flush_tile(const ChanArgs& p, int64_t c0, const float2* sI, float* accA, float* accB,
                           float* g_values, float* g_knots)
{
    __syncthreads();
    const int N = p.N;
    for (int e = threadIdx.x; e < (N + 1) * kCh; e += blockDim.x) {
        const int j = e / kCh, ch = e % kCh;
        const int64_t c = c0 + ch;
        if (c >= p.C) continue;
        const float A1 = (j < N) ? accA[(j + 1) * kCh + ch] : 0.0f;
        const float Bj = (j > 0) ? accB[j * kCh + ch] : 0.0f;
        float gv = A1 + Bj;
        if (j == 0) gv += accA[0 * kCh + ch];
        if (j == N) gv += accA[(N + 1) * kCh + ch];
        if (g_values && gv != 0.0f) atomicAdd(g_values + c * (int64_t)(N + 1) + j, gv);
        if (g_knots) {
            const float gk = -sI[(j + 1) * kCh + ch].x * A1 - sI[j * kCh + ch].x * Bj;
            if (gk != 0.0f) atomicAdd(g_knots + c * (int64_t)(N + 1) + j, gk);
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < (N + 2) * kCh; e += blockDim.x) {
        accA[e] = 0.0f;
        accB[e] = 0.0f;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kChThreads, 1) channels_backward_kernel(const ChanArgs p, const float* x,
                                                                          const float* gy, float* gx,
                                                                          float* g_values, float* g_knots)
{
    extern __shared__ float4 s_ch[];
    float2* sP = reinterpret_cast<float2*>(s_ch);
    float2* sI = sP + (size_t)p.K * kCh;
    float* accA = reinterpret_cast<float*>(sI + (size_t)(p.N + 2) * kCh);
    float* accB = accA + (size_t)(p.N + 2) * kCh;
    float* xs = accB + (size_t)(p.N + 2) * kCh;
    int* cj = reinterpret_cast<int*>(accA);  // build scratch aliases the accumulators
    __shared__ TileParams tp;
    const int64_t cluster = blockIdx.x >> 1, nclusters = gridDim.x >> 1;
    const int64_t u0 = p.units * cluster / nclusters, u1 = p.units * (cluster + 1) / nclusters;
    int64_t built = -1;
    for (int64_t u = u0; u < u1; ++u) {
        const int64_t tile = 2 * (u / p.per_pair) + (blockIdx.x & 1), chunk = u % p.per_pair;
        if (tile >= p.tiles) break;  // the odd tile out of an odd tile count
        if (tile != built) {
            if (built >= 0) flush_tile(p, built * kCh, sI, accA, accB, g_values, g_knots);
            __syncthreads();
            build_tile(p, tile * kCh, sP, sI, xs, cj, &tp);
            if (threadIdx.x == 0 && tp.bad) atomicOr(p.status, 1);
            for (int e = threadIdx.x; e < (p.N + 2) * kCh; e += blockDim.x) {
                accA[e] = 0.0f;
                accB[e] = 0.0f;
            }
            __syncthreads();
            built = tile;
        }
        const int64_t r0 = chunk * p.rows_per_unit, r1 = min(p.R, r0 + p.rows_per_unit);
        if (tp.any_chain)
            chan_bwd_rows<true>(p, tile * kCh, r0, r1, sP, sI, xs, tp, accA, accB, x, gy, gx);
        else
            chan_bwd_rows<false>(p, tile * kCh, r0, r1, sP, sI, xs, tp, accA, accB, x, gy, gx);
    }
    if (built >= 0) flush_tile(p, built * kCh, sI, accA, accB, g_values, g_knots);
}

}  // namespace

size_t channels_smem_bytes(int64_t N, int64_t K, bool backward)
{
    const size_t n1 = (size_t)(N + 1), n2 = (size_t)(N + 2);
    // forward: 8 channels of 16-byte cell records, knots, values, slopes and build scratch
    if (!backward) return sizeof(float4) * kChF * (size_t)K + 4 * sizeof(float) * kChF * n1;
    // backward: 16 channels of 8-byte cell and interval records, two accumulators, knots
    return sizeof(float2) * kCh * ((size_t)K + n2) + sizeof(float) * 2 * kCh * n2 + sizeof(float) * kCh * n1;
}

int64_t channels_default_cells(int64_t N, bool backward)
{
    // 4 (N+1) cells forward, 2 (N+1) backward, as far as one CTA's shared memory allows
    // the static tile parameters of the kernel share the CTA's shared memory
    const size_t budget = device_info().smem_optin - (backward ? sizeof(TileParams) : sizeof(TileParamsF));
    int64_t K = (backward ? 2 : 4) * (N + 1);
    while (K > 16 && channels_smem_bytes(N, K, backward) > budget) K -= 16;
    return K;
}

pwl_status channels_launch(const ChanArgs& base, bool backward, int io_dtype, const void* x, void* y,
                           const float* gy, float* gx, float* g_values, float* g_knots, cudaStream_t s)
{
    ChanArgs p = base;
    const size_t smem = channels_smem_bytes(p.N, p.K, backward);
    const DeviceInfo& di = device_info();
    const int tile_ch = backward ? kCh : kChF;       // channels per tile
    const int cluster_ctas = backward ? 2 : kClF;    // CTAs per cluster (adjacent tiles, same rows)
    if (smem + (backward ? sizeof(TileParams) : sizeof(TileParamsF)) > di.smem_optin)
        return fail(PWL_ENOTSUP, "channel index of %zu bytes (%d channels x %d cells, N = %d) does not fit one CTA",
                    smem, tile_ch, p.K, p.N);
    p.tiles = (p.C + tile_ch - 1) / tile_ch;
    const int64_t pairs = (p.tiles + cluster_ctas - 1) / cluster_ctas;  // tile groups of one cluster
    const void* kfn;
    if (backward)
        kfn = (const void*)channels_backward_kernel;
    else if (io_dtype == PWL_BF16)
        kfn = (const void*)channels_forward_kernel<__nv_bfloat16>;
    else
        kfn = (const void*)channels_forward_kernel<float>;
    PWL_CUDA_TRY(ensure_smem_limit(kfn, smem));
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster_ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kChThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3(cluster_ctas);
    int clusters = 0;
    PWL_CUDA_TRY(cudaOccupancyMaxActiveClusters(&clusters, kfn, &cfg));
    clusters = std::max(clusters, 1);
    // about 8 units per cluster: few index builds per CTA, and the last
    // units balance the load
    int64_t chunks = std::max<int64_t>(1, ((int64_t)clusters * 8 + pairs - 1) / pairs);
    chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, p.R / (kChThreads / tile_ch)));
    p.rows_per_unit = (p.R + chunks - 1) / chunks;
    chunks = (p.R + p.rows_per_unit - 1) / p.rows_per_unit;
    p.per_pair = chunks;
    p.units = pairs * chunks;
    clusters = (int)std::min<int64_t>(clusters, p.units);
    cfg.gridDim = dim3(cluster_ctas * clusters);
    if (backward) {
        PWL_CUDA_TRY(cudaLaunchKernelEx(&cfg, channels_backward_kernel, p, static_cast<const float*>(x), gy, gx,
                                        g_values, g_knots));
    } else if (io_dtype == PWL_BF16) {
        PWL_CUDA_TRY(cudaLaunchKernelEx(&cfg, channels_forward_kernel<__nv_bfloat16>, p,
                                        static_cast<const __nv_bfloat16*>(x), static_cast<__nv_bfloat16*>(y)));
    } else {
        PWL_CUDA_TRY(cudaLaunchKernelEx(&cfg, channels_forward_kernel<float>, p, static_cast<const float*>(x),
                                        static_cast<float*>(y)));
    }
    PWL_CHECK_LAUNCH("channels kernel");
    return PWL_OK;
}

}  // namespace pwl

using namespace pwl;

namespace {

pwl_status check_channels(const float* knots, const float* values, int64_t C, int64_t N, int64_t R,
                          int64_t k_cells, int32_t* d_status)
{
    if (!knots || !values) return fail(PWL_EINVAL, "knots / values is NULL");
    if (C < 1 || N < 1 || N > 65535) return fail(PWL_EINVAL, "need C >= 1 channels and 1 <= N <= 65535 intervals");
    if (R < 0) return fail(PWL_EINVAL, "rows must be >= 0");
    if (k_cells < 0 || k_cells > (1 << 20)) return fail(PWL_EINVAL, "k_cells must be in [0, 2^20]");
    if (!d_status) return fail(PWL_EINVAL, "status word is NULL");
    return PWL_OK;
}

}  // namespace

extern "C" {

pwl_status pwl_channels_forward(const float* d_knots, const float* d_values, int64_t n_channels,
                                int64_t n_intervals, int64_t k_cells, const void* d_x, void* d_y, int64_t rows,
                                int32_t io_dtype, int32_t* d_status, void* stream)
{
    clear_error();
    pwl_status st = check_channels(d_knots, d_values, n_channels, n_intervals, rows, k_cells, d_status);
    if (st != PWL_OK) return st;
    if (io_dtype != PWL_FP32 && io_dtype != PWL_BF16) return fail(PWL_EINVAL, "io dtype must be FP32 or BF16");
    if (rows == 0) return PWL_OK;
    if (!d_x || !d_y) return fail(PWL_EINVAL, "x / y is NULL");
    ChanArgs p{};
    p.knots = d_knots;
    p.values = d_values;
    p.C = n_channels;
    p.R = rows;
    p.N = (int)n_intervals;
    p.K = (int)(k_cells > 0 ? k_cells : channels_default_cells(n_intervals, false));
    p.status = d_status;
    return channels_launch(p, false, io_dtype, d_x, d_y, nullptr, nullptr, nullptr, nullptr, as_stream(stream));
}

pwl_status pwl_channels_backward(const float* d_knots, const float* d_values, int64_t n_channels,
                                 int64_t n_intervals, int64_t k_cells, const float* d_x, const float* d_gy,
                                 float* d_gx, float* d_g_values, float* d_g_knots, int64_t rows, int32_t* d_status,
                                 void* stream)
{
    clear_error();
    pwl_status st = check_channels(d_knots, d_values, n_channels, n_intervals, rows, k_cells, d_status);
    if (st != PWL_OK) return st;
    if (rows == 0) return PWL_OK;
    if (!d_x || !d_gy || !d_gx) return fail(PWL_EINVAL, "x / gy / gx is NULL");
    ChanArgs p{};
    p.knots = d_knots;
    p.values = d_values;
    p.C = n_channels;
    p.R = rows;
    p.N = (int)n_intervals;
    p.K = (int)(k_cells > 0 ? k_cells : channels_default_cells(n_intervals, true));
    p.status = d_status;
    return channels_launch(p, true, PWL_FP32, d_x, nullptr, d_gy, d_gx, d_g_values, d_g_knots, as_stream(stream));
}

}  // extern "C"
