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

// d_k for this thread's cells of the chunk at c0 (sum returned), THREADS
// threads per chunk; the sampled path is a template flag, chosen once per
// chunk
template <typename T, bool SAMPLED, int THREADS>
__device__ __forceinline__ double density_chunk(const pwl_func& F, int64_t c0, int64_t M, double delta,
                                                double* __restrict__ d)
{
    double acc = 0.0;
    for (int r = 0; r < kChunk / THREADS; ++r) {
        const int64_t k = c0 + r * THREADS + threadIdx.x;
        if (k < M) {
            // t_k = a + (k + 1/2) delta, rounded as written (no fused multiply-add)
            const double t = __dadd_rn(F.a, __dmul_rn((double)k + 0.5, delta));
            const T f2 = func_second_derivative_k<SAMPLED, T>(F, (T)t);
            const double dk = (double)FMath<T>::dens(f2);
            d[k] = dk;
            acc += dk;
        }
    }
    return acc;
}

// The density of a single function's few chunks (128 at N = 4096) takes
// kDensityThreads threads per chunk, so that its FP64 f'' evaluations keep
// more warps in flight per SM than the scans' 256-thread CTAs would: 512
// threads (the FP64 J0 path needs ~128 registers, so 1024 would spill
// heavily) took the bench's design graph of 9 tables from 0.56 to 0.49 ms.
constexpr int kDensityThreads = 512;

template <typename T, bool SAMPLED>
__global__ void __launch_bounds__(kDensityThreads) density_chunks_kernel(DesignPlan p)
{
    __shared__ double s_red[kDensityThreads / 32];
    for (int64_t ch = blockIdx.x; ch < p.total_chunks; ch += gridDim.x) {
        const int f = find_segment(p.choff, p.F, ch);
        const pwl_func F = p.funcs[f];
        if ((F.kind == PWL_F_SAMPLED) != SAMPLED) continue;  // the other launch's (uniform per CTA)
        const int64_t M = p.moff[f + 1] - p.moff[f];
        const int64_t c0 = (ch - p.choff[f]) * kChunk;
        const double delta = (F.b - F.a) / (double)M;
        double* __restrict__ d = p.d + p.moff[f];
        double acc = density_chunk<T, SAMPLED, kDensityThreads>(F, c0, M, delta, d);
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < kDensityThreads / 32; ++w) s += s_red[w];
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

// ---- fused design of whole functions (batches) ----------------------------
// One CTA designs one function at a time, in one launch for the batch:
//   pass A  for every 2048-cell chunk: the densities (8 contiguous cells per
//           thread), the chunk total (block scan in FP64) and the chunk's
//           last cell of positive density;
//   scan    exclusive FP64 scan of the chunk totals: chunk bases, G_M;
//   pass B  for every chunk holding targets tau_i (G at the chunk start <=
//           tau_i < G at the next chunk's start): the densities again, the
//           FP64 prefix of the thread partials, and for each such knot the
//           largest cell k with G_k <= tau_i (binary search over the thread
//           prefixes, then the thread's cells), the walk back to a cell of
//           positive density, and x_i = a + k delta + (tau_i - G_k) / d_k.
// Nothing per cell goes to memory.  Thread partials of 8 densities are a
// plain FP64 sum (FP64 mode) or a compensated FP32 sum (FP32 mode: two-sum,
// every rounding error carried, about 2^-48 relative); all sums above them
// are FP64.  In FP32 mode the cell midpoints are formed in FP32 from the
// chunk start (the FP32 f'' rounds its argument to FP32 anyway).
template <typename T>
struct Partial;
template <>
struct Partial<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s = __dadd_rn(s, v); }
    __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Partial<float> {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v)
    {
        const float t = __fadd_rn(s, v);
        const float bp = __fsub_rn(t, s);
        const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
        s = t;
        c = __fadd_rn(c, e);
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// The uncompensated running sum of a partial, in the density's type: the
// cheap candidate of the in-thread cell search (checked in FP64 after).
__device__ __forceinline__ double approx(const Partial<double>& p) { return p.s; }
__device__ __forceinline__ float approx(const Partial<float>& p) { return p.s; }

// FP64 density of cell k: |f''(t_k)|^{2/5}, t_k = a + (k + 1/2) delta
template <bool SAMPLED>
__device__ __forceinline__ double fused_density64(const pwl_func& F, double a, double delta, int64_t k)
{
    const double t = __dadd_rn(a, __dmul_rn((double)k + 0.5, delta));
    return pow_two_fifths(func_second_derivative_k<SAMPLED, double>(F, t));
}

// The densities of one chunk's cells of this thread, added to `part`; STORE
// keeps them in s_d, LAST tracks the last cell of positive density.  The
// sampled path is a template flag, chosen once per chunk.
template <bool SAMPLED, bool STORE, bool LAST>
__device__ __forceinline__ void fused_chunk64(const pwl_func& F, double a, double delta, int64_t c0, int cnt,
                                              Partial<double>& part, int& last, double* s_d)
{
    for (int r = 0; r < kPerThread; ++r) {
        const int l = threadIdx.x * kPerThread + r;
        if (l < cnt) {
            const double dk = fused_density64<SAMPLED>(F, a, delta, c0 + l);
            if (STORE) s_d[l] = dk;
            part.add(dk);
            if (LAST && dk > 0.0) last = l;
        }
    }
}
// FP32 density from the function's FP32 constants: |f''|^{2/5} by the
// hardware exp2/log2 pair (__powf), a few ulp (the FP32 mode's knot bound
// allows a relative density error near 1e-6), for a third of the
// instructions of powf
template <bool SAMPLED>
__device__ __forceinline__ float fused_density_f(const FuncF& G, const pwl_func& F, float t0f, float deltaf,
                                                 int local)
{
    const float t = __fmaf_rn((float)local + 0.5f, deltaf, t0f);
    float f2;
    if constexpr (SAMPLED) f2 = (float)sampled_second_derivative(F, (double)t);
    else f2 = func_second_derivative_f(G, t);
    return __powf(fabsf(f2), 0.4f);
}


// smallest i in [1, N] with tau_i = i G_M / N >= G (N if none below N)
__device__ __forceinline__ int64_t first_target_at_or_above(double G, double GM, int64_t N)
{
    auto tau = [&](int64_t i) { return (double)i * GM / (double)N; };
    const double e = floor(G / GM * (double)N);
    int64_t i = (int64_t)fmin(fmax(e, 1.0), (double)N);
    while (i > 1 && tau(i - 1) >= G) --i;
    while (i < N && tau(i) < G) ++i;
    return i;
}

template <typename T, bool SAMPLED>
__global__ void __launch_bounds__(kDesignThreads) design_fused_kernel(DesignPlan p)
{
    __shared__ T s_d[kChunk];
    __shared__ double s_S[kDesignThreads];  // chunk base + exclusive prefix of the thread partials
    __shared__ double s_G[kDesignThreads];  // delta * s_S: G at each thread's first cell
    __shared__ double s_warp[kDesignThreads / 32 + 1];
    __shared__ int s_last;
    const int t = threadIdx.x;
    for (int o = blockIdx.x; o < p.F; o += gridDim.x) {
        const int f = p.order[o];
        const pwl_func F = p.funcs[f];
        if ((F.kind == PWL_F_SAMPLED) != SAMPLED) continue;  // the other launch's (uniform per CTA)
        const int64_t M = p.moff[f + 1] - p.moff[f];
        const int64_t N = p.koff[f + 1] - p.koff[f] - 1;
        const int64_t nch = p.choff[f + 1] - p.choff[f];
        const double a = F.a, b = F.b;
        const double delta = (b - a) / (double)M;
        const float deltaf = (float)delta;
        double* __restrict__ knots = p.knots + p.koff[f];
        double* __restrict__ csum = p.csum + p.choff[f];
        double* __restrict__ cbase = p.cbase + p.choff[f];
        int* __restrict__ clast = p.clast + p.choff[f];

        // pass A
        for (int64_t ch = 0; ch < nch; ++ch) {
            const int64_t c0 = ch * kChunk;
            const int cnt = (int)min((int64_t)kChunk, M - c0);
            const float t0f = (float)(a + (double)c0 * delta);
            Partial<T> part;
            int last = -1;
            fused_chunk64<SAMPLED, false, true>(F, a, delta, c0, cnt, part, last, nullptr);
            if (t == 0) s_last = -1;
            __syncthreads();
            if (last >= 0) atomicMax(&s_last, last);
            double tot;
            block_exclusive_scan(part.value(), s_warp, &tot);
            if (t == 0) {
                csum[ch] = tot;
                clast[ch] = s_last;
            }
        }
        __syncthreads();
        // exclusive scan of the chunk totals
        double carry = 0.0;
        for (int64_t base = 0; base < nch; base += kDesignThreads) {
            const int64_t c = base + t;
            const double v = c < nch ? csum[c] : 0.0;
            double tot;
            const double ex = block_exclusive_scan(v, s_warp, &tot);
            if (c < nch) cbase[c] = carry + ex;
            carry += tot;
        }
        __syncthreads();
        const double GM = delta * carry;
        if (t == 0) {
            knots[0] = a;
            knots[N] = b;
        }
        if (!(GM > 0.0)) {  // f linear on I (or no finite density): the uniform partition
            for (int64_t i = 1 + t; i < N; i += kDesignThreads) knots[i] = a + (double)i * (b - a) / (double)N;
            __syncthreads();
            continue;
        }
        // the first target of every chunk, all chunks at once (the chunk sums
        // are spent: their area takes the indices)
        int64_t* ifirst = reinterpret_cast<int64_t*>(csum);
        for (int64_t c = t; c < nch; c += kDesignThreads) ifirst[c] = first_target_at_or_above(delta * cbase[c], GM, N);
        __syncthreads();

        // pass B
        int64_t lastpos = -1;  // last cell of positive density before the current chunk
        for (int64_t ch = 0; ch < nch; ++ch) {
            const int64_t c0 = ch * kChunk;
            const int64_t i0 = ifirst[ch], i1 = ch + 1 < nch ? ifirst[ch + 1] : N;
            if (i0 < i1) {
                const int cnt = (int)min((int64_t)kChunk, M - c0);
                const float t0f = (float)(a + (double)c0 * delta);
                Partial<T> part;
                int unused = -1;
                fused_chunk64<SAMPLED, true, false>(F, a, delta, c0, cnt, part, unused, s_d);
                double tot;
                const double ex = block_exclusive_scan(part.value(), s_warp, &tot);
                s_S[t] = cbase[ch] + ex;
                s_G[t] = delta * (cbase[ch] + ex);
                __syncthreads();
                const int U = (cnt + kPerThread - 1) / kPerThread;  // threads holding cells
                // G at local cell l: delta * (S_u + partial of the thread's cells before l)
                auto g_at = [&](int l) {
                    const int u = l / kPerThread;
                    Partial<T> q;
                    for (int r = u * kPerThread; r < l; ++r) q.add(s_d[r]);
                    return delta * (s_S[u] + q.value());
                };
                const double inv_delta = 1.0 / delta;
                for (int64_t i = i0 + t; i < i1; i += kDesignThreads) {
                    const double tau = (double)i * GM / (double)N;
                    int lo = 0, hi = U - 1;  // largest u with G at its first cell <= tau (u = 0 is)
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_G[mid] <= tau) lo = mid; else hi = mid - 1;
                    }
                    // largest cell r of thread lo with G_r <= tau: a candidate from
                    // the running sums in T against tau / delta - S, then the exact
                    // FP64 G of the candidate and its right neighbour decide
                    const int nr = min(kPerThread, cnt - lo * kPerThread);
                    const T target = (T)(tau * inv_delta - s_S[lo]);
                    Partial<T> run;
                    int r = 0;
                    for (int q = 1; q < nr; ++q) {
                        run.add(s_d[lo * kPerThread + q - 1]);
                        if (approx(run) <= target) r = q;
                    }
                    int kl = lo * kPerThread + r;
                    double Gk = g_at(kl);
                    while (kl > lo * kPerThread && !(Gk <= tau)) Gk = g_at(--kl);
                    while (kl + 1 < lo * kPerThread + nr) {
                        const double Gn = g_at(kl + 1);
                        if (!(Gn <= tau)) break;
                        ++kl;
                        Gk = Gn;
                    }
                    int kk = kl;  // largest cell <= kl of positive density
                    while (kk >= 0 && !(s_d[kk] > T(0))) --kk;
                    double x;
                    if (kk >= 0) {
                        if (kk != kl) Gk = g_at(kk);
                        const double dk = (double)s_d[kk];
                        x = __dadd_rn(a, __dmul_rn((double)(c0 + kk), delta));
                        const double step = fmin(fmax((tau - Gk) / dk, 0.0), delta);
                        x = __dadd_rn(x, step);
                    } else if (lastpos >= 0) {
                        // no density from cell lastpos + 1 to here, so tau is at or past
                        // G at the end of cell lastpos: its right edge
                        x = __dadd_rn(__dadd_rn(a, __dmul_rn((double)lastpos, delta)), delta);
                    } else {
                        x = a;  // no positive density from the start of I
                    }
                    knots[i] = x;
                }
            }
            const int cl = clast[ch];
            if (cl >= 0) lastpos = c0 + cl;
            __syncthreads();  // s_d and s_S are rewritten for the next chunk
        }
    }
}

// ---- fused design, FP32 mode ------------------------------------------------
// The FP32-density variant of design_fused_kernel, arranged so that almost
// no FP64 operation is spent per density cell (GB300 runs about one FP64
// operation per SM and cycle):
//   - pass A writes the FP32 densities to scratch; pass B reads them back;
//   - sums inside a chunk are float-float (a compensated pair hi + lo, about
//     48 significant bits): thread partials, the block scan and the chunk
//     total; the chunk totals, their scan and G_M are FP64;
//   - the knot search compares float-float values in FP32, in units of the
//     density sum (G / delta): the target tau_i / delta = i G_M / (N delta)
//     minus the chunk base is formed in FP64 once per knot and split into a
//     float-float pair;
//   - the step inside the cell, (tau_i - G_k) / d_k, is FP32 (it is at most
//     delta, so its rounding is below 1e-7 delta), and x = a + k delta + step
//     is FP64.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF x, FF y)
{
    const float s = __fadd_rn(x.hi, y.hi);
    const float bp = __fsub_rn(s, x.hi);
    const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bp)), __fsub_rn(y.hi, bp));
    const float t = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
    const float hi = __fadd_rn(s, t);
    return FF{hi, __fsub_rn(t, __fsub_rn(hi, s))};
}
__device__ __forceinline__ FF ff_neg(FF x) { return FF{-x.hi, -x.lo}; }
__device__ __forceinline__ bool ff_le(FF x, FF y) { return x.hi < y.hi || (x.hi == y.hi && x.lo <= y.lo); }
__device__ __forceinline__ FF ff_from_double(double v)
{
    const float hi = __double2float_rn(v);
    return FF{hi, __double2float_rn(v - (double)hi)};
}
__device__ __forceinline__ double ff_to_double(FF x) { return (double)x.hi + (double)x.lo; }

// Block-wide exclusive scan of one float-float per thread (kDesignThreads);
// *total receives the block sum.
__device__ __forceinline__ FF ff_block_exclusive_scan(FF v, FF* s_w, FF* total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int W = kDesignThreads / 32;
    FF incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const FF n{__shfl_up_sync(0xffffffffu, incl.hi, o), __shfl_up_sync(0xffffffffu, incl.lo, o)};
        if (lane >= o) incl = ff_add(n, incl);
    }
    FF excl{__shfl_up_sync(0xffffffffu, incl.hi, 1), __shfl_up_sync(0xffffffffu, incl.lo, 1)};
    if (lane == 0) excl = FF{0.0f, 0.0f};
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        FF ws = lane < W ? s_w[lane] : FF{0.0f, 0.0f};
        FF wi = ws;
        for (int o = 1; o < W; o <<= 1) {
            const FF n{__shfl_up_sync(0xffffffffu, wi.hi, o), __shfl_up_sync(0xffffffffu, wi.lo, o)};
            if (lane >= o) wi = ff_add(n, wi);
        }
        FF we{__shfl_up_sync(0xffffffffu, wi.hi, 1), __shfl_up_sync(0xffffffffu, wi.lo, 1)};
        if (lane == 0) we = FF{0.0f, 0.0f};
        if (lane < W) s_w[lane] = we;
        if (lane == W - 1) s_w[W] = wi;
    }
    __syncthreads();
    const FF r = ff_add(s_w[warp], excl);
    *total = s_w[W];
    __syncthreads();
    return r;
}

// Block-wide float-float sum (kDesignThreads); the result is valid in
// thread 0.  One barrier.
__device__ __forceinline__ FF ff_block_sum(FF v, FF* s_w)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1)
        v = ff_add(v, FF{__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)});
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    FF r{0.0f, 0.0f};
    if (threadIdx.x == 0)
        for (int w = 0; w < kDesignThreads / 32; ++w) r = ff_add(r, s_w[w]);
    return r;
}

// smallest i in [1, N] with i c >= S (N if none below N), c = G_M / (N delta)
__device__ __forceinline__ int64_t first_target_at_or_above_units(double S, double c, int64_t N)
{
    const double e = floor(S / c);
    int64_t i = (int64_t)fmin(fmax(e, 1.0), (double)N);
    while (i > 1 && (double)(i - 1) * c >= S) --i;
    while (i < N && (double)i * c < S) ++i;
    return i;
}

// The densities of one chunk into scratch, with the float-float total of the
// thread's cells and its last cell of positive density.  Sampled functions
// take a loop of their own, so that their FP64 interpolation does not weigh
// on the registers of the analytic kinds' loop.
template <bool SAMPLED>
__device__ __forceinline__ void chunk_densities_f(const FuncF& G, const pwl_func& F, float t0f, float deltaf,
                                                  int cnt, float* __restrict__ dchunk, FF& part, int& last)
{
    for (int r = 0; r < kPerThread; ++r) {
        const int l = threadIdx.x * kPerThread + r;
        if (l < cnt) {
            const float dk = fused_density_f<SAMPLED>(G, F, t0f, deltaf, l);
            dchunk[l] = dk;
            part = ff_add(part, FF{dk, 0.0f});
            if (dk > 0.0f) last = l;
        }
    }
}

template <bool SAMPLED>
__global__ void __launch_bounds__(kDesignThreads, 4) design_fused_fp32_kernel(DesignPlan p)
{
    __shared__ float s_d[kChunk];
    __shared__ FF s_ex[kDesignThreads];  // exclusive float-float prefix of the thread partials
    __shared__ FF s_w[2 * (kDesignThreads / 32) + 1];
    __shared__ int s_last2[2];
    __shared__ double s_warp[kDesignThreads / 32 + 1];
    __shared__ int s_last;
    const int t = threadIdx.x;
    float* __restrict__ dbuf_all = reinterpret_cast<float*>(p.d);
    if (t < 2) s_last2[t] = -1;
    __syncthreads();
    for (int o = blockIdx.x; o < p.F; o += gridDim.x) {
        const int f = p.order[o];
        const pwl_func F = p.funcs[f];
        if ((F.kind == PWL_F_SAMPLED) != SAMPLED) continue;  // the other launch's (uniform per CTA)
        const FuncF G = make_funcf(F);  // FP32 constants of f'', once per function
        const int64_t M = p.moff[f + 1] - p.moff[f];
        const int64_t N = p.koff[f + 1] - p.koff[f] - 1;
        const int64_t nch = p.choff[f + 1] - p.choff[f];
        const double a = F.a, b = F.b;
        const double delta = (b - a) / (double)M;
        const float deltaf = (float)delta;
        double* __restrict__ knots = p.knots + p.koff[f];
        double* __restrict__ csum = p.csum + p.choff[f];
        double* __restrict__ cbase = p.cbase + p.choff[f];
        int* __restrict__ clast = p.clast + p.choff[f];
        float* __restrict__ dbuf = dbuf_all + p.moff[f];

        // pass A: densities (to scratch), chunk totals, last positive cell
        for (int64_t ch = 0; ch < nch; ++ch) {
            const int64_t c0 = ch * kChunk;
            const int cnt = (int)min((int64_t)kChunk, M - c0);
            const float t0f = (float)(a + (double)c0 * delta);
            FF part{0.0f, 0.0f};
            int last = -1;
            chunk_densities_f<SAMPLED>(G, F, t0f, deltaf, cnt, dbuf + c0, part, last);
            // chunk total and last positive cell: one barrier per chunk (the
            // slot pair alternates so that a chunk's writes never meet the
            // previous chunk's reads)
            const int slot = (int)(ch & 1);
            if (last >= 0) atomicMax(&s_last2[slot], last);
            const FF tot = ff_block_sum(part, s_w + slot * (kDesignThreads / 32));
            if (t == 0) {
                csum[ch] = ff_to_double(tot);
                clast[ch] = s_last2[slot];
                s_last2[slot] = -1;
            }
        }
        __syncthreads();
        double carry = 0.0;
        for (int64_t base = 0; base < nch; base += kDesignThreads) {
            const int64_t c = base + t;
            const double v = c < nch ? csum[c] : 0.0;
            double tot;
            const double ex = block_exclusive_scan(v, s_warp, &tot);
            if (c < nch) cbase[c] = carry + ex;
            carry += tot;
        }
        __syncthreads();
        const double GM = delta * carry;
        if (t == 0) {
            knots[0] = a;
            knots[N] = b;
        }
        if (!(GM > 0.0)) {
            for (int64_t i = 1 + t; i < N; i += kDesignThreads) knots[i] = a + (double)i * (b - a) / (double)N;
            __syncthreads();
            continue;
        }
        const double cunit = carry / (double)N;  // tau_i / delta = i * cunit
        // the first target of every chunk, all chunks at once (the chunk sums
        // are spent: their area takes the indices)
        int64_t* ifirst = reinterpret_cast<int64_t*>(csum);
        for (int64_t c = t; c < nch; c += kDesignThreads) ifirst[c] = first_target_at_or_above_units(cbase[c], cunit, N);
        __syncthreads();

        // pass B
        int64_t lastpos = -1;
        for (int64_t ch = 0; ch < nch; ++ch) {
            const int64_t c0 = ch * kChunk;
            const int64_t i0 = ifirst[ch], i1 = ch + 1 < nch ? ifirst[ch + 1] : N;
            if (i0 < i1) {
                const int cnt = (int)min((int64_t)kChunk, M - c0);
                FF part{0.0f, 0.0f};
                for (int r = 0; r < kPerThread; ++r) {
                    const int l = t * kPerThread + r;
                    if (l < cnt) {
                        const float dk = dbuf[c0 + l];
                        s_d[l] = dk;
                        part = ff_add(part, FF{dk, 0.0f});
                    }
                }
                FF tot;
                s_ex[t] = ff_block_exclusive_scan(part, s_w, &tot);
                __syncthreads();
                const int U = (cnt + kPerThread - 1) / kPerThread;
                const double cb = cbase[ch];
                // float-float prefix of local cell l: S_u + the thread's cells before l
                auto ff_at = [&](int l) {
                    const int u = l / kPerThread;
                    FF q = s_ex[u];
                    for (int r = u * kPerThread; r < l; ++r) q = ff_add(q, FF{s_d[r], 0.0f});
                    return q;
                };
                for (int64_t i = i0 + t; i < i1; i += kDesignThreads) {
                    const FF tl = ff_from_double((double)i * cunit - cb);  // target in the chunk
                    int lo = 0, hi = U - 1;  // largest u with S_u <= target (u = 0 is)
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (ff_le(s_ex[mid], tl)) lo = mid; else hi = mid - 1;
                    }
                    const int nr = min(kPerThread, cnt - lo * kPerThread);
                    FF q = s_ex[lo], Sk = q;
                    int kl = lo * kPerThread;
                    for (int r = 1; r < nr; ++r) {
                        q = ff_add(q, FF{s_d[lo * kPerThread + r - 1], 0.0f});
                        if (!ff_le(q, tl)) break;
                        kl = lo * kPerThread + r;
                        Sk = q;
                    }
                    int kk = kl;
                    while (kk >= 0 && !(s_d[kk] > 0.0f)) --kk;
                    double x;
                    if (kk >= 0) {
                        if (kk != kl) Sk = ff_at(kk);
                        const FF diff = ff_add(tl, ff_neg(Sk));  // (tau - G_k) / delta
                        const float step = fminf(fmaxf((diff.hi + diff.lo) * deltaf / s_d[kk], 0.0f), deltaf);
                        x = __dadd_rn(__fma_rn((double)(c0 + kk), delta, a), (double)step);
                    } else if (lastpos >= 0) {
                        x = __dadd_rn(__dadd_rn(a, __dmul_rn((double)lastpos, delta)), delta);
                    } else {
                        x = a;
                    }
                    knots[i] = x;
                }
            }
            const int cl = clast[ch];
            if (cl >= 0) lastpos = c0 + cl;
            __syncthreads();
        }
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
    const int kinds = plan_kinds(p.kinds);
    if (kinds & kKindsAnalytic) {
        if (p.precision == PWL_PREC_FP32)
            density_chunks_kernel<float, false><<<grid_chunks, kDensityThreads, 0, s>>>(p);
        else
            density_chunks_kernel<double, false><<<grid_chunks, kDensityThreads, 0, s>>>(p);
        PWL_CHECK_LAUNCH("density_chunks_kernel");
    }
    if (kinds & kKindsSampled) {
        if (p.precision == PWL_PREC_FP32)
            density_chunks_kernel<float, true><<<grid_chunks, kDensityThreads, 0, s>>>(p);
        else
            density_chunks_kernel<double, true><<<grid_chunks, kDensityThreads, 0, s>>>(p);
        PWL_CHECK_LAUNCH("density_chunks_kernel");
    }
    chunk_scan_kernel<<<(int)std::min<int64_t>(p.F, 65535), kDesignThreads, 0, s>>>(p);
    PWL_CHECK_LAUNCH("chunk_scan_kernel");
    cumulative_kernel<<<grid_chunks, kDesignThreads, 0, s>>>(p);
    PWL_CHECK_LAUNCH("cumulative_kernel");
    const int grid_knots = (int)std::min<int64_t>((p.total_knots + 255) / 256, (int64_t)di.sms * 16);
    invert_kernel<<<grid_knots, 256, 0, s>>>(p);
    PWL_CHECK_LAUNCH("invert_kernel");
    return PWL_OK;
}

pwl_status design_fused_launch(const DesignPlan& p, cudaStream_t s)
{
    const DeviceInfo& di = device_info();
    const int grid = (int)std::min<int64_t>(p.F, (int64_t)di.sms * 8);
    const int kinds = plan_kinds(p.kinds);
    if (kinds & kKindsAnalytic) {
        if (p.precision == PWL_PREC_FP32)
            design_fused_fp32_kernel<false><<<grid, kDesignThreads, 0, s>>>(p);
        else
            design_fused_kernel<double, false><<<grid, kDesignThreads, 0, s>>>(p);
        PWL_CHECK_LAUNCH("design_fused_kernel");
    }
    if (kinds & kKindsSampled) {
        if (p.precision == PWL_PREC_FP32)
            design_fused_fp32_kernel<true><<<grid, kDesignThreads, 0, s>>>(p);
        else
            design_fused_kernel<double, true><<<grid, kDesignThreads, 0, s>>>(p);
        PWL_CHECK_LAUNCH("design_fused_kernel");
    }
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
    p.kinds = kinds_of(f, 1);
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
