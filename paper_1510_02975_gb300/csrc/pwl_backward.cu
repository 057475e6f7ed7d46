// pwl_backward.cu -- gradients of Algorithm 1 w.r.t. the query x, the
// vertex values v_j and the knots x_j.
//
// With interval i of x, h = x_i - x_{i-1}, delta = (x - x_{i-1})/h and slope s:
//   dy/dx = s,  dy/dv_{i-1} = 1 - delta,  dy/dv_i = delta,
//   dy/dx_{i-1} = -s (1 - delta),  dy/dx_i = -s delta.
// Because s is constant on an interval, the table gradients only need two
// sums per interval, A_i = sum gy (1 - delta) and B_i = sum gy delta:
//   g_v[j]  += A_{j+1} + B_j            g_x[j] += -s_{j+1} A_{j+1} - s_j B_j
// (clamped queries add gy to g_v[0] or g_v[N] only).
//
// Pass 1 (persistent grid): every CTA stages the backward records (in up to
// 8 bank-private copies) and the reciprocal lengths, streams (x, gy) -> gx
// with 16-byte vectors, and accumulates A, B in shared memory: per-lane
// atomics into up to 32 accumulator copies for random queries, a warp-level
// sum for vectors that lie in one or two intervals (sorted or clustered
// queries), and registers for a warp's hot interval (a point mass) and for
// the queries beyond the ends of [a, b] and at x = b (x = a is interval 1 at
// delta = 0, an interior query).  It then writes its partial sums to the
// workspace (one row per CTA).
// The shared-memory sums are 32-bit fixed point (FP32 shared-memory atomic
// adds are a compare-and-swap loop in software; 32-bit integer adds are a
// single native operation, ~4x the throughput with random bins).  Each CTA
// picks its unit 2^-F from the geometric mean of the |gy| in its first
// vectors, so that a typical term is ~2^22 units; a term t = rint(c 2^F)
// then carries an absolute error of at most half a unit.  The int32 adds
// wrap modulo 2^32, and the lane whose add wraps (seen from the old value
// the atomic returns: exactly one lane per wrap) adds +-2^32 units to the
// CTA's row in global memory, so every sum is exact in integer arithmetic
// whatever the order of the adds.  A term of 2^31 units or more adds its low
// 32 bits the same way and its multiple of 2^32 units to the row (exact in
// FP32 while the row holds fewer than 2^24 such multiples); only terms
// beyond 2^62 units, inf and NaN are summed in FP32 (global FP32
// reductions are native).
// Pass 2: 32 knots per CTA, the CTA rows split over 16 thread groups, sums
// the rows in a fixed order (FP64) and forms g_v and g_x.  The in-CTA
// integer sums and the wraps (multiples of 2^32 units) do not depend on the
// order of the adds; only the FP32 terms of a row (clamped queries, x = b,
// terms beyond the int32 range) do, so results without those are
// reproducible bit for bit, the rest to the rounding of those terms.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "pwl_backward.cuh"

namespace pwl {

namespace {

constexpr int kBwdUnroll = 2;

// Accumulator layout per CTA row (2 (N + 2) entries; int32 fixed point in
// shared memory, FP32 in the row):
//   A[0]      gy of queries clamped on the left  -> g_v[0]
//   A[1..N]   sum gy (1 - delta) on interval i
//   A[N+1]    gy of queries clamped on the right -> g_v[N]
//   B[0..N+1] sum gy delta on interval i (entries 0 and N+1 unused)
struct BwdArgs {
    const float4* rec;  // backward records {x_j, j, s_j, s_{j+1} | link} or {x_j, j | inside, 1/h_{j+1}, s_{j+1}}
    const TableHeader* hdr;
    const float* inv_h;
    const float* slope;
    int N, K, n_smem, max_chain;
    int lanes;          // accumulator copies (a power of two <= 32), lane l adds into copy l mod lanes
    int rep_shift;      // log2 of the record copies R: lane l reads srec[c R + l mod R]
    float a, b, inv_w, off;
    float s_last;       // slope of interval N (set by the kernel)
    int64_t nvec;       // float4 vectors (x, gy and gx all 16-byte aligned), else 0
    // set by the kernel: the CTA's fixed-point unit 2^-F (scale = 2^F), the
    // value of one int32 wrap (2^(32-F)) and the CTA's row (A columns at
    // rowA, B columns at rowB = rowA + N + 2)
    float scale, wrap;
    float* rowA;
    float* rowB;
};

// Fixed-point add of a scaled term vs = v 2^F of any size: T = rint(vs) as
// a 64-bit integer is split into its low 32 bits r (signed), added to the
// shared accumulator, and q = (T - r) / 2^32, which goes with the wrap of
// that add (if any) to the row as q 2^(32-F) (a multiple of 2^32 units:
// FP32 sums such multiples exactly while the row holds fewer than 2^24 of
// them).  Terms beyond 2^62 units, inf and NaN go to the row as FP32.
__device__ __forceinline__ void fix_add_wide(int* acc, float* grow, float vs, float v, float wrap)
{
    if (fabsf(vs) < 0x1p62f) {
        const long long T = __float2ll_rn(vs);
        const int r = (int)(unsigned)(unsigned long long)T;
        long long q = (T - (long long)r) >> 32;
        const int old = atomicAdd(acc, r);
        const int nw = (int)((unsigned)old + (unsigned)r);
        if (((old ^ nw) & ~(old ^ r)) < 0) q += r < 0 ? -1 : 1;
        if (q != 0) atomicAdd(grow, (float)q * wrap);
    } else {
        atomicAdd(grow, v);
    }
}

// The common case of fix_add_wide: |vs| < 2^31, one native atomic, a wrap
// reported to the row as +-2^(32-F).
__device__ __forceinline__ void fix_add(int* acc, float* grow, float vs, float v, float wrap)
{
    if (fabsf(vs) < 0x1p31f) {
        const int t = __float2int_rn(vs);
        const int old = atomicAdd(acc, t);
        const int nw = (int)((unsigned)old + (unsigned)t);
        if (((old ^ nw) & ~(old ^ t)) < 0) atomicAdd(grow, t < 0 ? -wrap : wrap);
    } else {
        fix_add_wide(acc, grow, vs, v, wrap);
    }
}

// Queries beyond the ends of [a, b] and at x = b all feed the same three
// sums; a skewed input (a query set clipped to the domain) can send half of
// them there, so they are summed in registers and added once per warp at
// the end instead of through contended shared-memory atomics.
struct EndSums {
    float clamped_left, clamped_right, at_b;
};

// One query, without branches apart from chain walks: the lookup runs on the
// clamped point (a NaN looks up a and contributes nothing), the interval and
// the side come from selects.  A query in [a, b) returns its interval in
// `bin` and its two sums gy (1 - delta), gy delta in ca, cb; any other query
// returns bin = -1 (the ends are summed in registers).
template <bool CHAINS, bool STAGED>
__device__ __forceinline__ float bwd_query(float x, float g, const float4* __restrict__ srec,
                                           const float* __restrict__ s_ih, EndSums& e, const BwdArgs& p, int& bin,
                                           float& ca, float& cb)
{
    const float xc = fminf(fmaxf(x, p.a), p.b);  // NaN -> a
    const int c = cell_of(xc, p.inv_w, p.off, p.K);
    float4 r = (STAGED || c < p.n_smem) ? srec[c << p.rep_shift] : __ldg(p.rec + c);
    if (CHAINS) {
        for (int it = 0; it < p.max_chain && xc >= r.x && is_link(r.w); ++it) {
            const int j = link_index(r.w);
            r = (STAGED || j < p.n_smem) ? srec[j << p.rep_shift] : __ldg(p.rec + j);
        }
    }
    const uint32_t jy = __float_as_uint(r.y);
    const bool inside = (jy & kInsideFlag) != 0;  // knot-free cell: 1/h_{j+1} in r.z
    const int j = (int)(jy & ~kInsideFlag);
    // left of x_j: interval j, measured from its right end; else interval
    // j + 1 (an interior query never reaches x_N, where j + 1 would be N + 1)
    const bool lside = !inside && xc < r.x;
    const int i = lside ? j : j + 1;
    const float s = lside ? r.z : r.w;
    float ih = r.z;
    if (!inside) ih = s_ih[i];  // knot cells only: the shared gather of 1/h_i
    const float tt = (lside ? (r.x - xc) : (xc - r.x)) * ih;
    const float delta = lside ? 1.0f - tt : tt;
    const float one_minus = lside ? tt : 1.0f - tt;
    bin = i;
    ca = g * one_minus;
    cb = g * delta;
    float gx = g * s;
    // x = a needs nothing apart: its lookup is interval 1 at delta = 0 (the
    // hot-interval registers absorb a point mass there, as in a set clipped
    // to the domain)
    if (!(x >= p.a && x < p.b)) {  // beyond the ends, x = b, NaN: rare in most query sets
        bin = -1;
        // clamped queries feed g_v[0] or g_v[N]; x = b is interval N at delta = 1
        e.clamped_left += x < p.a ? g : 0.0f;
        e.clamped_right += x > p.b ? g : 0.0f;
        e.at_b += x == p.b ? g : 0.0f;
        gx = x == p.b ? g * p.s_last : 0.0f;
        gx = x != x ? x : gx;
    }
    return gx;
}

// A query's two sums into its lane's accumulator copy: both terms share the
// range check (|ca| + |cb| = |gy|); the rare query outside it takes the wide
// path for both
__device__ __forceinline__ void bwd_scatter(int* accA, int* accB, int bin, float ca, float cb, const BwdArgs& p,
                                            int copy)
{
    const float sa = ca * p.scale, sb = cb * p.scale;
    if (bin >= 0 && fabsf(sa) + fabsf(sb) < 0x1p31f) {
        const int ta = __float2int_rn(sa), tb = __float2int_rn(sb);
        const int oa = atomicAdd(accA + bin * p.lanes + copy, ta);
        const int ob = atomicAdd(accB + bin * p.lanes + copy, tb);
        // sign bit of w: old + t left the int32 range (one branch for both)
        const int wa = (oa ^ (int)((unsigned)oa + (unsigned)ta)) & ~(oa ^ ta);
        const int wb = (ob ^ (int)((unsigned)ob + (unsigned)tb)) & ~(ob ^ tb);
        if ((wa | wb) < 0) {
            if (wa < 0) atomicAdd(p.rowA + bin, ta < 0 ? -p.wrap : p.wrap);
            if (wb < 0) atomicAdd(p.rowB + bin, tb < 0 ? -p.wrap : p.wrap);
        }
    } else if (bin >= 0) {
        fix_add_wide(accA + bin * p.lanes + copy, p.rowA + bin, sa, ca, p.wrap);
        fix_add_wide(accB + bin * p.lanes + copy, p.rowB + bin, sb, cb, p.wrap);
    }
}

template <bool CHAINS, bool STAGED>
__device__ __forceinline__ float bwd_one(float x, float g, const float4* __restrict__ srec,
                                         const float* __restrict__ s_ih, int* accA, int* accB,
                                         EndSums& e, const BwdArgs& p, int copy)
{
    int bin;
    float ca, cb;
    const float gx = bwd_query<CHAINS, STAGED>(x, g, srec, s_ih, e, p, bin, ca, cb);
    bwd_scatter(accA, accB, bin, ca, cb, p, copy);
    return gx;
}

// Whether every query of the warp's vector (four per lane, 128 in all) is
// interior and lies in the interval of the warp's first query (bF) or of its
// last (bL).  The first vote, on one query per lane, fails at once for random
// queries; both votes are warp-uniform.
__device__ __forceinline__ bool warp_two_bins(const int (&bin)[4], int& bF, int& bL)
{
    bF = __shfl_sync(0xffffffffu, bin[0], 0);
    bL = __shfl_sync(0xffffffffu, bin[3], 31);
    if (!__all_sync(0xffffffffu, bin[0] >= 0 && (bin[0] == bF || bin[0] == bL))) return false;
    bool ok = true;
#pragma unroll
    for (int k = 1; k < 4; ++k) ok = ok && bin[k] >= 0 && (bin[k] == bF || bin[k] == bL);
    return __all_sync(0xffffffffu, ok);
}

// A warp's hot interval (warp-uniform; -1: none) and this lane's sums A, B
// for it, kept in registers instead of shared-memory atomics.
struct HotBin {
    int bin;
    float a, b;
};

// lanes (of 32) that must share lane 0's interval on a detection vote for the
// interval to become the warp's hot one
constexpr int kHotLanes = 8;

// The hot interval's sums into shared memory (warp-uniform call: every lane
// of the warp runs it)
__device__ __forceinline__ void flush_hot(int* accA, int* accB, HotBin& h, const BwdArgs& p, int lane)
{
    if (h.bin < 0) return;
    for (int o = 16; o > 0; o >>= 1) {
        h.a += __shfl_xor_sync(0xffffffffu, h.a, o);
        h.b += __shfl_xor_sync(0xffffffffu, h.b, o);
    }
    if (lane == 0) {
        fix_add(accA + h.bin * p.lanes, p.rowA + h.bin, h.a * p.scale, h.a, p.wrap);
        fix_add(accB + h.bin * p.lanes, p.rowB + h.bin, h.b * p.scale, h.b, p.wrap);
    }
    h.a = 0.0f;
    h.b = 0.0f;
}

// A query's sums: into the hot interval's registers, or the lane's copy
__device__ __forceinline__ void bwd_scatter_hot(int* accA, int* accB, int bin, float ca, float cb,
                                                const BwdArgs& p, int copy, HotBin& h)
{
    const bool hit = bin == h.bin;
    h.a += hit ? ca : 0.0f;
    h.b += hit ? cb : 0.0f;
    bwd_scatter(accA, accB, hit ? -1 : bin, ca, cb, p, copy);
}

// Four consecutive queries per lane, 128 per warp, all 32 lanes active.
// Warp-aggregated scatter-add for sorted or clustered queries, where per-lane
// atomics would all hit one or two addresses and serialise: when the whole
// vector lies in intervals bF and bL, the warp sums the two intervals' A and
// B by shuffles and lanes 0 and 1 add them with four atomics.  A warp runs in
// one of two modes (`agg`, warp-uniform).  Per lane: each query's atomics
// are issued right after its lookup, and on `detect` vectors one ballot on
// the lanes' first queries against lane 0's interval decides: all 32 lanes
// in it switch to the aggregated mode; kHotLanes or more make it the warp's
// hot interval (a point mass scattered through the stream, which no vector
// aggregates: its queries' sums then stay in registers).  Aggregated: the
// vector's lookups come first, and a vector that spans more intervals falls
// back to per-lane atomics and switches back.
template <bool CHAINS, bool STAGED>
__device__ __forceinline__ float4 bwd_vec_warp(float4 xv, float4 gv, const float4* __restrict__ srec,
                                               const float* __restrict__ s_ih, int* accA, int* accB,
                                               EndSums& e, const BwdArgs& p, int copy, int lane, bool detect,
                                               bool& agg, HotBin& hot)
{
    int bin[4], bF, bL;
    float4 o;
    if (!agg) {
        float ca, cb;
        if (hot.bin < 0) {
            o.x = bwd_query<CHAINS, STAGED>(xv.x, gv.x, srec, s_ih, e, p, bin[0], ca, cb);
            bwd_scatter(accA, accB, bin[0], ca, cb, p, copy);
            o.y = bwd_query<CHAINS, STAGED>(xv.y, gv.y, srec, s_ih, e, p, bin[1], ca, cb);
            bwd_scatter(accA, accB, bin[1], ca, cb, p, copy);
            o.z = bwd_query<CHAINS, STAGED>(xv.z, gv.z, srec, s_ih, e, p, bin[2], ca, cb);
            bwd_scatter(accA, accB, bin[2], ca, cb, p, copy);
            o.w = bwd_query<CHAINS, STAGED>(xv.w, gv.w, srec, s_ih, e, p, bin[3], ca, cb);
            bwd_scatter(accA, accB, bin[3], ca, cb, p, copy);
        } else {
            o.x = bwd_query<CHAINS, STAGED>(xv.x, gv.x, srec, s_ih, e, p, bin[0], ca, cb);
            bwd_scatter_hot(accA, accB, bin[0], ca, cb, p, copy, hot);
            o.y = bwd_query<CHAINS, STAGED>(xv.y, gv.y, srec, s_ih, e, p, bin[1], ca, cb);
            bwd_scatter_hot(accA, accB, bin[1], ca, cb, p, copy, hot);
            o.z = bwd_query<CHAINS, STAGED>(xv.z, gv.z, srec, s_ih, e, p, bin[2], ca, cb);
            bwd_scatter_hot(accA, accB, bin[2], ca, cb, p, copy, hot);
            o.w = bwd_query<CHAINS, STAGED>(xv.w, gv.w, srec, s_ih, e, p, bin[3], ca, cb);
            bwd_scatter_hot(accA, accB, bin[3], ca, cb, p, copy, hot);
        }
        if (detect) {
            const int b0 = __shfl_sync(0xffffffffu, bin[0], 0);
            const unsigned same = __ballot_sync(0xffffffffu, bin[0] >= 0 && bin[0] == b0);
            agg = same == 0xffffffffu;
            if (!agg && b0 != hot.bin && __popc(same) >= kHotLanes) {
                flush_hot(accA, accB, hot, p, lane);
                hot.bin = b0;
            }
        }
        return o;
    }
    float ca[4], cb[4];
    o.x = bwd_query<CHAINS, STAGED>(xv.x, gv.x, srec, s_ih, e, p, bin[0], ca[0], cb[0]);
    o.y = bwd_query<CHAINS, STAGED>(xv.y, gv.y, srec, s_ih, e, p, bin[1], ca[1], cb[1]);
    o.z = bwd_query<CHAINS, STAGED>(xv.z, gv.z, srec, s_ih, e, p, bin[2], ca[2], cb[2]);
    o.w = bwd_query<CHAINS, STAGED>(xv.w, gv.w, srec, s_ih, e, p, bin[3], ca[3], cb[3]);
    agg = warp_two_bins(bin, bF, bL);
    if (agg) {
        float aF = 0.0f, bFs = 0.0f, aL = 0.0f, bLs = 0.0f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool f = bin[k] == bF;
            aF += f ? ca[k] : 0.0f;
            bFs += f ? cb[k] : 0.0f;
            aL += f ? 0.0f : ca[k];
            bLs += f ? 0.0f : cb[k];
        }
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
            aF += __shfl_xor_sync(0xffffffffu, aF, o2);
            bFs += __shfl_xor_sync(0xffffffffu, bFs, o2);
            aL += __shfl_xor_sync(0xffffffffu, aL, o2);
            bLs += __shfl_xor_sync(0xffffffffu, bLs, o2);
        }
        if (lane == 0) {
            fix_add(accA + bF * p.lanes, p.rowA + bF, aF * p.scale, aF, p.wrap);
            fix_add(accB + bF * p.lanes, p.rowB + bF, bFs * p.scale, bFs, p.wrap);
        } else if (lane == 1 && bL != bF) {
            const int c1 = 1 & (p.lanes - 1);
            fix_add(accA + bL * p.lanes + c1, p.rowA + bL, aL * p.scale, aL, p.wrap);
            fix_add(accB + bL * p.lanes + c1, p.rowB + bL, bLs * p.scale, bLs, p.wrap);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) bwd_scatter(accA, accB, bin[k], ca[k], cb[k], p, copy);
    }
    return o;
}

template <bool CHAINS, bool STAGED>
__device__ __forceinline__ void backward_body(const BwdArgs& p, const float4* __restrict__ srec,
                                              const float* __restrict__ s_ih, int* accA, int* accB,
                                              EndSums& e, const float* x, const float* gy, float* gx, int64_t m)
{
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int copy = threadIdx.x & (p.lanes - 1);
    const float4* xv = reinterpret_cast<const float4*>(x);
    const float4* gv = reinterpret_cast<const float4*>(gy);
    float4* ov = reinterpret_cast<float4*>(gx);
    int64_t i = tid;
    bool agg = true;
    HotBin hot{-1, 0.0f, 0.0f};
    // warp-uniform bound (the warp's last lane decides), so that the whole
    // warp runs these iterations and their votes together
    for (; i + (31 - lane) + (kBwdUnroll - 1) * nthr < p.nvec; i += kBwdUnroll * nthr) {
        float4 xs[kBwdUnroll], gs[kBwdUnroll];
#pragma unroll
        for (int u = 0; u < kBwdUnroll; ++u) {
            xs[u] = __ldcs(xv + i + u * nthr);
            gs[u] = __ldcs(gv + i + u * nthr);
        }
#pragma unroll
        for (int u = 0; u < kBwdUnroll; ++u)
            __stcs(ov + i + u * nthr, bwd_vec_warp<CHAINS, STAGED>(xs[u], gs[u], srec, s_ih, accA, accB, e, p, copy, lane,
                                                               u == kBwdUnroll - 1, agg, hot));
    }
    for (; i < p.nvec; i += nthr) {
        const float4 xs = __ldcs(xv + i), gs = __ldcs(gv + i);
        float4 o;
        o.x = bwd_one<CHAINS, STAGED>(xs.x, gs.x, srec, s_ih, accA, accB, e, p, copy);
        o.y = bwd_one<CHAINS, STAGED>(xs.y, gs.y, srec, s_ih, accA, accB, e, p, copy);
        o.z = bwd_one<CHAINS, STAGED>(xs.z, gs.z, srec, s_ih, accA, accB, e, p, copy);
        o.w = bwd_one<CHAINS, STAGED>(xs.w, gs.w, srec, s_ih, accA, accB, e, p, copy);
        __stcs(ov + i, o);
    }
    for (int64_t q = p.nvec * 4 + tid; q < m; q += nthr)
        gx[q] = bwd_one<CHAINS, STAGED>(x[q], gy[q], srec, s_ih, accA, accB, e, p, copy);
    flush_hot(accA, accB, hot, p, lane);  // every lane of the warp gets here
}

// The CTA's fixed-point unit comes from the mean binary exponent of the
// nonzero finite |gy| among the first vector of each of its threads (a
// geometric mean, so that a few outliers do not coarsen the unit of the
// typical terms): F = kFixTypicalBits - that mean, so a typical term is
// ~2^22 units.  exponent_stats adds the binary exponent of a nonzero finite
// |g| to esum and counts it in ecnt (zero, subnormal, inf and NaN are
// skipped); with no usable value F = kFixTypicalBits.  F stays inside
// [-60, 126]: 2^F and 2^-F are normal FP32 numbers, and a term of the wide
// path (below 2^62 units) carries at most 2^30 multiples of 2^(32-F), which
// stays below FP32's largest value.  Gradients whose typical magnitude is
// below 2^-103 (~1e-31) therefore get a unit coarser than 2^-23 of them.
constexpr int kFixTypicalBits = 23;
__device__ __forceinline__ void exponent_stats(float g, int& esum, int& ecnt)
{
    const uint32_t e = (__float_as_uint(g) >> 23) & 0xffu;
    const bool ok = e != 0u && e != 0xffu;
    esum += ok ? (int)e - 127 : 0;
    ecnt += ok ? 1 : 0;
}
__device__ __forceinline__ int fix_exponent(int esum, int ecnt)
{
    const int e_mean = ecnt > 0 ? (int)floorf((float)esum / (float)ecnt) : 0;
    return min(max(kFixTypicalBits - e_mean, -60), 126);
}
__device__ __forceinline__ float exp2_int(int e) { return __int_as_float((e + 127) << 23); }

__global__ void __launch_bounds__(1024) backward_kernel(const BwdArgs args, const float* x, const float* gy,
                                                        float* gx, int64_t m, float* partials)
{
    extern __shared__ float4 s_dyn[];
    const int R = 1 << args.rep_shift;
    // this lane's record copy: srec[c << rep_shift] is copy (lane mod R) of record c
    const float4* srec = s_dyn + (threadIdx.x & (R - 1));
    float* s_ih = reinterpret_cast<float*>(s_dyn + (size_t)args.n_smem * R);
    int* accA = reinterpret_cast<int*>(s_ih + (args.N + 2));
    int* accB = accA + (size_t)(args.N + 2) * args.lanes;
    int* s_exp = accB + (size_t)(args.N + 2) * args.lanes;  // exponent sum and count
    BwdArgs p = args;
    const int W = 2 * (p.N + 2);
    float* row = partials + (size_t)blockIdx.x * W;
    p.rowA = row;
    p.rowB = row + (p.N + 2);
    if (threadIdx.x == 0) s_exp[0] = s_exp[1] = 0;
    const int n_chain = p.hdr->n_chain_b;
    p.max_chain = p.hdr->max_chain_b;
    p.n_smem = min(p.K + n_chain, p.n_smem);
    p.s_last = p.slope[p.N];
    for (int i = threadIdx.x; i < (p.n_smem << p.rep_shift); i += blockDim.x)
        s_dyn[i] = __ldg(p.rec + (i >> p.rep_shift));
    for (int i = threadIdx.x; i < p.N + 2; i += blockDim.x) s_ih[i] = p.inv_h[i];
    for (int i = threadIdx.x; i < W * p.lanes; i += blockDim.x) accA[i] = 0;
    // the row collects the FP32 terms and the wraps during the pass
    for (int i = threadIdx.x; i < W; i += blockDim.x) row[i] = 0.0f;
    int esum = 0, ecnt = 0;
    {
        // the first vector (or query) this thread will process (read at the
        // L2, not through the read-only path: gx may alias gy)
        const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (p.nvec > 0) {
            if (tid < p.nvec) {
                const float4 g4 = __ldcg(reinterpret_cast<const float4*>(gy) + tid);
                exponent_stats(g4.x, esum, ecnt);
                exponent_stats(g4.y, esum, ecnt);
                exponent_stats(g4.z, esum, ecnt);
                exponent_stats(g4.w, esum, ecnt);
            }
        } else if (tid < m) {
            exponent_stats(__ldcg(gy + tid), esum, ecnt);
        }
    }
    esum = __reduce_add_sync(0xffffffffu, esum);
    ecnt = __reduce_add_sync(0xffffffffu, ecnt);
    __syncthreads();  // s_exp zeroed, staging done
    if ((threadIdx.x & 31) == 0 && ecnt > 0) {
        atomicAdd(&s_exp[0], esum);
        atomicAdd(&s_exp[1], ecnt);
    }
    __syncthreads();
    const int F = fix_exponent(s_exp[0], s_exp[1]);
    p.scale = exp2_int(F);          // 2^F
    p.wrap = exp2_int(32 - F);      // 2^(32-F)
    const float unit = exp2_int(-F);  // 2^-F
    EndSums e{0.0f, 0.0f, 0.0f};
    // every record in shared memory (the usual case): no global-record branch per lookup
    const bool staged = p.n_smem >= p.K + n_chain;
    if (n_chain == 0) {
        if (staged) backward_body<false, true>(p, srec, s_ih, accA, accB, e, x, gy, gx, m);
        else backward_body<false, false>(p, srec, s_ih, accA, accB, e, x, gy, gx, m);
    } else {
        if (staged) backward_body<true, true>(p, srec, s_ih, accA, accB, e, x, gy, gx, m);
        else backward_body<true, false>(p, srec, s_ih, accA, accB, e, x, gy, gx, m);
    }
    for (int o = 16; o > 0; o >>= 1) {
        e.clamped_left += __shfl_xor_sync(0xffffffffu, e.clamped_left, o);
        e.clamped_right += __shfl_xor_sync(0xffffffffu, e.clamped_right, o);
        e.at_b += __shfl_xor_sync(0xffffffffu, e.at_b, o);
    }
    if ((threadIdx.x & 31) == 0) {  // FP32 terms of the row
        if (e.clamped_left != 0.0f) atomicAdd(p.rowA, e.clamped_left);
        if (e.clamped_right != 0.0f) atomicAdd(p.rowA + p.N + 1, e.clamped_right);
        if (e.at_b != 0.0f) atomicAdd(p.rowB + p.N, e.at_b);
    }
    __syncthreads();  // every shared add and every FP32 add to the row done
    // entry k of the row: its copies summed in 64-bit integers (thread k
    // starts at copy k mod L, so that a warp's reads spread over the banks),
    // times 2^-F, plus the FP32 terms and wraps gathered in the row (read at
    // the L2, where the reductions were performed)
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
        long long v = 0;
        const int* a = accA + (size_t)k * p.lanes;
        for (int c = 0; c < p.lanes; ++c) v += a[(c + k) & (p.lanes - 1)];
        row[k] = __fmaf_rn((float)v, unit, __ldcg(row + k));
    }
}

// g_v[j] += A_{j+1} + B_j (+ clamped terms), g_x[j] += -s_{j+1} A_{j+1} - s_j B_j.
// A CTA covers kRedKnots consecutive knots; its kRedGroups warps-worth of
// threads split the partial-sum rows (thread group g takes rows g, g + G, ...;
// coalesced 128-byte reads per row), and group 0 adds the groups' FP64 sums
// in a fixed order, so the result does not depend on scheduling.  Column j+1
// of a row is A_{j+1} (j = N: the right-clamped sum), column N+2+j is B_j
// (j = 0: column 0, the left-clamped sum), so g_v[j] is always the sum of
// the two columns.
constexpr int kRedKnots = 32, kRedGroups = 16;

__global__ void __launch_bounds__(kRedKnots * kRedGroups)
    backward_reduce_kernel(const float* __restrict__ partials, int rows, int N, const float* __restrict__ slope,
                           float* g_values, float* g_knots)
{
    __shared__ double s_a[kRedGroups][kRedKnots], s_b[kRedGroups][kRedKnots];
    const int lane = threadIdx.x % kRedKnots, grp = threadIdx.x / kRedKnots;
    const int j = blockIdx.x * kRedKnots + lane;
    const size_t W = 2 * (size_t)(N + 2);
    double a = 0.0, b = 0.0;
    if (j <= N) {
        const float* colA = partials + (j + 1);
        const float* colB = partials + (j == 0 ? 0 : N + 2 + j);
        int r = grp;
        for (; r + 3 * kRedGroups < rows; r += 4 * kRedGroups) {
            float va[4], vb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                va[u] = __ldg(colA + (size_t)(r + u * kRedGroups) * W);
                vb[u] = __ldg(colB + (size_t)(r + u * kRedGroups) * W);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a += (double)va[u];
                b += (double)vb[u];
            }
        }
        for (; r < rows; r += kRedGroups) {
            a += (double)__ldg(colA + (size_t)r * W);
            b += (double)__ldg(colB + (size_t)r * W);
        }
    }
    s_a[grp][lane] = a;
    s_b[grp][lane] = b;
    __syncthreads();
    if (grp != 0 || j > N) return;
    for (int g = 1; g < kRedGroups; ++g) {
        a += s_a[g][lane];
        b += s_b[g][lane];
    }
    if (g_values) g_values[j] += (float)(a + b);
    if (g_knots) {
        double gk = 0.0;
        if (j < N) gk -= (double)slope[j + 1] * a;
        if (j > 0) gk -= (double)slope[j] * b;
        g_knots[j] += (float)gk;
    }
}

}  // namespace

BwdShape backward_shape(pwl_table t)
{
    BwdShape s{};
    s.err = cudaSuccess;
    s.n_smem = backward_smem_records(t);
    if (s.n_smem < 0) return s;
    s.smem = backward_smem_bytes(t);
    s.threads = 1024;
    s.err = occupancy_grid(backward_kernel, s.threads, s.smem, &s.grid);
    if (s.err != cudaSuccess) {
        s.n_smem = -1;
        return s;
    }
    s.workspace = sizeof(float) * 2 * (size_t)(t->N + 2) * (size_t)s.grid;
    return s;
}

pwl_status backward_launch(pwl_table t, const float* x, const float* gy, float* gx, float* g_values,
                           float* g_knots, int64_t m, float* partials, int grid, cudaStream_t s)
{
    const BwdShape sh = backward_shape(t);
    BwdArgs p{};
    p.rec = t->rec_b;
    p.hdr = t->hdr;
    p.inv_h = t->inv_h;
    p.slope = t->slope;
    p.N = (int)t->N;
    p.K = (int)t->Kb;
    p.n_smem = (int)sh.n_smem;
    p.max_chain = 0;
    p.lanes = backward_lanes(t);
    p.rep_shift = 0;
    while ((1 << p.rep_shift) < backward_record_copies(t)) ++p.rep_shift;
    p.a = t->a;
    p.b = t->b;
    p.inv_w = t->inv_w_b;
    p.off = t->off_b;
    const uintptr_t ax = reinterpret_cast<uintptr_t>(x), ag = reinterpret_cast<uintptr_t>(gy),
                    ao = reinterpret_cast<uintptr_t>(gx);
    p.nvec = ((ax | ag | ao) % 16 == 0) ? m / 4 : 0;
    backward_kernel<<<grid, sh.threads, sh.smem, s>>>(p, x, gy, gx, m, partials);
    PWL_CHECK_LAUNCH("backward_kernel");
    if (g_values || g_knots) {
        backward_reduce_kernel<<<(int)((t->N + kRedKnots) / kRedKnots), kRedKnots * kRedGroups, 0, s>>>(
            partials, grid, (int)t->N, t->slope, g_values, g_knots);
        PWL_CHECK_LAUNCH("backward_reduce_kernel");
    }
    return PWL_OK;
}

// ---------------------------------------------------------------------------
// Backward without any allocation: the per-CTA partial sums live in a
// fixed, file-scope device array instead of a caller workspace.
// ---------------------------------------------------------------------------
namespace {

// 2^21 floats (8 MiB) per GPU that loads the library, held until exit.
constexpr size_t kStaticPartials = (size_t)1 << 21;
static __device__ __align__(256) float g_static_partials[kStaticPartials];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
float* g_static_addr[kMaxDevices] = {};

// Device address of g_static_partials on `dev` (the current device).  The
// first call per device looks it up; in host code the array's name is only
// a host-side stand-in, never a device address.
pwl_status static_partials(int dev, float** out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(PWL_ENOTSUP, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_partials)");
        g_static_addr[dev] = static_cast<float*>(p);
    }
    *out = g_static_addr[dev];
    return PWL_OK;
}

}  // namespace

}  // namespace pwl

using namespace pwl;

extern "C" {

pwl_status pwl_eval_backward_noalloc(pwl_table t, const float* d_x, const float* d_gy, float* d_gx,
                                     float* d_g_values, float* d_g_knots, int64_t m, void* stream)
{
    clear_error();
    if (!t) return fail(PWL_EINVAL, "table is NULL");
    if (m < 0) return fail(PWL_EINVAL, "m must be >= 0");
    if (m > 0 && (!d_x || !d_gy || !d_gx)) return fail(PWL_EINVAL, "x / gy / gx is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return fail(PWL_EINVAL, "table lives on device %d, current device is %d", t->device, dev);
    // device_info() of this device is already cached: pwl_table_build used it
    const BwdShape sh = backward_shape(t);
    if (sh.n_smem < 0) {
        if (sh.err != cudaSuccess) return cuda_fail(sh.err, "backward kernel launch shape");
        return fail(PWL_ENOTSUP, "backward stages 12 (N+2) bytes of shared memory; N = %lld is too large",
                    (long long)t->N);
    }
    const int sms = device_info().sms;
    const int64_t row = 2 * (t->N + 2);
    const int64_t rows = (int64_t)(kStaticPartials / (size_t)row);
    if (rows < sms)
        return fail(PWL_EINVAL,
                    "N = %lld too large for the static scratch of %zu floats: it needs one row of 2 (N + 2) "
                    "floats per SM, so N <= %lld on this %d-SM GPU",
                    (long long)t->N, kStaticPartials, (long long)(kStaticPartials / (2 * (size_t)sms)) - 2, sms);
    float* partials = nullptr;
    pwl_status st = static_partials(dev, &partials);
    if (st != PWL_OK) return st;
    if (m == 0) return PWL_OK;
    const int64_t units = m / 4 + 1;
    int64_t grid = std::min<int64_t>(sh.grid, rows);
    grid = std::min<int64_t>(grid, std::max<int64_t>(1, (units + sh.threads - 1) / sh.threads));
    // every launched CTA overwrites its whole row before the reduction reads
    // it, so the array's leftover contents from earlier calls do not matter
    return backward_launch(t, d_x, d_gy, d_gx, d_g_values, d_g_knots, m, partials, (int)grid,
                           as_stream(stream));
}

size_t pwl_eval_backward_workspace_size(pwl_table t)
{
    if (!t) return 0;
    return backward_shape(t).workspace;
}

pwl_status pwl_eval_backward(pwl_table t, const float* d_x, const float* d_gy, float* d_gx,
                             float* d_g_values, float* d_g_knots, int64_t m, void* d_workspace,
                             size_t workspace_bytes, void* stream)
{
    clear_error();
    if (!t) return fail(PWL_EINVAL, "table is NULL");
    if (m < 0) return fail(PWL_EINVAL, "m must be >= 0");
    if (m > 0 && (!d_x || !d_gy || !d_gx)) return fail(PWL_EINVAL, "x / gy / gx is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != t->device) return fail(PWL_EINVAL, "table lives on device %d, current device is %d", t->device, dev);
    const BwdShape sh = backward_shape(t);
    if (sh.n_smem < 0) {
        if (sh.err != cudaSuccess) return cuda_fail(sh.err, "backward kernel launch shape");
        return fail(PWL_ENOTSUP, "backward stages 12 (N+2) bytes of shared memory; N = %lld is too large",
                    (long long)t->N);
    }
    if (!d_workspace || workspace_bytes < sh.workspace)
        return fail(PWL_EINVAL, "workspace of %zu bytes needed (got %zu)", sh.workspace, workspace_bytes);
    if (m == 0) return PWL_OK;
    const int64_t units = m / 4 + 1;
    const int grid = (int)std::min<int64_t>(sh.grid, std::max<int64_t>(1, (units + sh.threads - 1) / sh.threads));
    return backward_launch(t, d_x, d_gy, d_gx, d_g_values, d_g_knots, m, static_cast<float*>(d_workspace),
                           grid, as_stream(stream));
}

}  // extern "C"
