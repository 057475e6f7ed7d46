// pwl_common.cuh -- internal declarations shared by the libpwl translation
// units: error reporting, device properties, the analytic test functions,
// the device table layout and the uniform cell index.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "pwl.h"
#include "pwl_bessel.cuh"

namespace pwl {

// ---------------------------------------------------------------------------
// host-side error handling
// ---------------------------------------------------------------------------
pwl_status fail(pwl_status s, const char* fmt, ...);
pwl_status cuda_fail(cudaError_t e, const char* what);
void clear_error();

#define PWL_CUDA_TRY(expr)                                              \
    do {                                                                \
        cudaError_t e_ = (expr);                                        \
        if (e_ != cudaSuccess) return ::pwl::cuda_fail(e_, #expr);      \
    } while (0)

#define PWL_CHECK_LAUNCH(what)                                          \
    do {                                                                \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return ::pwl::cuda_fail(e_, what);       \
    } while (0)

struct DeviceInfo {
    int device;
    int sms;
    size_t smem_optin;   // max dynamic shared memory per block (opt-in)
    size_t smem_per_sm;  // shared memory per multiprocessor
    int max_threads_sm;
};
// properties of the current device (cached per device)
const DeviceInfo& device_info();
// Raises a kernel's dynamic shared-memory limit to at least smem (never
// lowers it), and the persistent grid of a kernel (resident CTAs per SM
// times the SM count) with that limit set; both cached per device and kernel.
cudaError_t ensure_smem_limit(const void* fn, size_t smem);
cudaError_t occupancy_grid_fn(const void* fn, int threads, size_t smem, int* grid);
template <typename Kern>
inline cudaError_t raise_smem_limit(Kern kern, size_t smem)
{
    return ensure_smem_limit(reinterpret_cast<const void*>(kern), smem);
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Every device allocation of the library goes through these, so that a test
// can make them fail (pwl_test_fail_allocations) and see each call that
// allocates return PWL_ENOMEM and release what it had taken.
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_malloc_array(cudaArray_t* a, const cudaChannelFormatDesc* d, size_t width);

// ---------------------------------------------------------------------------
// analytic functions: f and f'' (FP64 and FP32 versions)
// ---------------------------------------------------------------------------
// |x|^{2/5} in FP64, the knot density of Eq. 16.  Newton's iteration for the
// inverse fifth root of a^2 (a = |x|): w -> w + w (1 - a^2 w^5) / 5 converges
// quadratically to a^{-2/5} (error e -> ~3 e^2).  Started from an FP32
// estimate (relative error ~3e-6), two steps reach FP64 rounding, and then
// a^2 w^4 = a^{2/5}: ~16 FP64 operations, no division.  Arguments outside
// [1e-30, 1e30] (zero, NaN, infinity, extreme magnitudes) go to pow.
__device__ __forceinline__ double pow_two_fifths(double x)
{
    const double a = fabs(x);
    if (!(a >= 1e-30 && a <= 1e30)) return pow(a, 0.4);
    double w = (double)exp2f(-0.4f * __log2f((float)a));
    const double a2 = a * a;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double w2 = w * w;
        const double e = fma(-(a2 * (w2 * w2)), w, 1.0);
        w = fma(w * e, 0.2, w);
    }
    const double w2 = w * w;
    return a2 * (w2 * w2);
}

template <typename T>
struct FMath;
template <>
struct FMath<double> {
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
    static __device__ __forceinline__ double bj0(double x) { return bessel_j0(x); }
    static __device__ __forceinline__ double bj1(double x) { return bessel_j1(x); }
    static __device__ __forceinline__ double dens(double x) { return pow_two_fifths(x); }
};
template <>
struct FMath<float> {
    static __device__ __forceinline__ float ex(float x) { return expf(x); }
    static __device__ __forceinline__ float bj0(float x) { return bessel_j0(x); }
    static __device__ __forceinline__ float bj1(float x) { return bessel_j1(x); }
    static __device__ __forceinline__ float dens(float x) { return powf(fabsf(x), 0.4f); }
};

// PWL_F_SAMPLED: p[0] = S, p[1] = the 64 bits of the samples' address
__host__ __device__ __forceinline__ uint64_t sampled_address(const pwl_func& F)
{
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(F.p[1]);  // a register move: F stays in registers
#else
    uint64_t a;
    memcpy(&a, &F.p[1], sizeof(a));
    return a;
#endif
}

// The sampled function's cell: u = (x - a)/h (as x - a times 1/h, p[3]),
// j = min(max(floor(u), 1), S - 3).  No division on the device: h, 1/h and
// 1/h^2 are in the descriptor (p[2..4], written by pwl_func_sampled).
struct SampledCell {
    const double* s;
    int64_t j;
    double t;  // u - j, in [-1, 2] after the clamp (the end cells extrapolate)
    double inv_h2;
};
__device__ __forceinline__ SampledCell sampled_cell(const pwl_func& F, double x)
{
    const int64_t S = (int64_t)F.p[0];
    const double u = (x - F.a) * F.p[3];
    const double fu = floor(u);
    const int64_t j = fu < 1.0 ? 1 : (fu > (double)(S - 3) ? S - 3 : (int64_t)fu);
    SampledCell c;
    c.s = reinterpret_cast<const double*>(sampled_address(F));
    c.j = j;
    c.t = u - (double)j;
    c.inv_h2 = F.p[4];
    return c;
}
// f: the cubic through samples j-1 .. j+2 (Lagrange form, nodes -1, 0, 1, 2)
__device__ __forceinline__ double sampled_value(const pwl_func& F, double x)
{
    const SampledCell c = sampled_cell(F, x);
    const double t = c.t;
    const double* s = c.s + c.j;
    const double lm = -t * (t - 1.0) * (t - 2.0) / 6.0;
    const double l0 = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
    const double l1 = -(t + 1.0) * t * (t - 2.0) / 2.0;
    const double l2 = (t + 1.0) * t * (t - 1.0) / 6.0;
    return lm * s[-1] + l0 * s[0] + l1 * s[1] + l2 * s[2];
}
// f'': second differences at samples j and j+1, linearly interpolated
__device__ __forceinline__ double sampled_second_derivative(const pwl_func& F, double x)
{
    const SampledCell c = sampled_cell(F, x);
    const double* s = c.s + c.j;
    const double dj = (s[-1] - 2.0 * s[0] + s[1]) * c.inv_h2;
    const double dk = (s[0] - 2.0 * s[1] + s[2]) * c.inv_h2;
    return dj + c.t * (dk - dj);
}

// f(x) for the analytic kinds of pwl_kind.
template <typename T>
__device__ __forceinline__ T func_value_analytic(const pwl_func& F, T x)
{
    using M = FMath<T>;
    switch (F.kind) {
    case PWL_F_GAUSSIAN: {
        T u = (x - (T)F.p[1]) / (T)F.p[2];
        return (T)F.p[0] * M::ex(T(-0.5) * u * u);
    }
    case PWL_F_LORENTZIAN: {
        T u = (x - (T)F.p[1]) / (T)F.p[2];
        return (T)F.p[0] / (T(1) + u * u);
    }
    case PWL_F_BESSEL_J0:
        return (T)F.p[0] * M::bj0((T)F.p[1] * x);
    case PWL_F_POLY: {
        T s = T(0);
        for (int k = 7; k >= 0; --k) s = s * x + (T)F.p[k];
        return s;
    }
    case PWL_F_EXP:
        return (T)F.p[0] * M::ex((T)F.p[1] * x);
    }
    return T(0);
}

// f''(x): Gaussian A (u^2-1)/s^2 e^{-u^2/2}; Lorentzian A (6u^2-2)/(g^2 (1+u^2)^3);
// J0(alpha x): A alpha^2 (J1(z)/z - J0(z)) (Bessel's equation, limit 1/2 at 0);
// polynomial and exponential by direct differentiation.
template <typename T>
__device__ __forceinline__ T func_second_derivative_analytic(const pwl_func& F, T x)
{
    using M = FMath<T>;
    switch (F.kind) {
    case PWL_F_GAUSSIAN: {
        T s = (T)F.p[2];
        T u = (x - (T)F.p[1]) / s;
        return (T)F.p[0] * (u * u - T(1)) / (s * s) * M::ex(T(-0.5) * u * u);
    }
    case PWL_F_LORENTZIAN: {
        T g = (T)F.p[2];
        T u = (x - (T)F.p[1]) / g;
        T q = T(1) + u * u;
        return (T)F.p[0] * (T(6) * u * u - T(2)) / (g * g * q * q * q);
    }
    case PWL_F_BESSEL_J0: {
        T al = (T)F.p[1];
        T z = al * x;
        T b0, b1;
        bessel_j01(z, b0, b1);
        T r = (fabs(z) < T(1e-8)) ? T(0.5) - z * z / T(16) : b1 / z;
        return (T)F.p[0] * al * al * (r - b0);
    }
    case PWL_F_POLY: {
        T s = T(0);
        for (int k = 7; k >= 2; --k) s = s * x + (T)(k * (k - 1)) * (T)F.p[k];
        return s;
    }
    case PWL_F_EXP:
        return (T)F.p[0] * (T)F.p[1] * (T)F.p[1] * M::ex((T)F.p[1] * x);
    }
    return T(0);
}

// f and f'' of any kind, the sampled path chosen at compile time: hot loops
// pick the instantiation once per function (or interval), so that the FP64
// interpolation of sampled functions adds no registers to the analytic kinds'
// loops; f and f'' choose at run time where that does not matter.
template <bool SAMPLED, typename T>
__device__ __forceinline__ T func_value_k(const pwl_func& F, T x)
{
    if constexpr (SAMPLED) return (T)sampled_value(F, (double)x);
    else return func_value_analytic<T>(F, x);
}
template <bool SAMPLED, typename T>
__device__ __forceinline__ T func_second_derivative_k(const pwl_func& F, T x)
{
    if constexpr (SAMPLED) return (T)sampled_second_derivative(F, (double)x);
    else return func_second_derivative_analytic<T>(F, x);
}
template <typename T>
__device__ __forceinline__ T func_value(const pwl_func& F, T x)
{
    return F.kind == PWL_F_SAMPLED ? func_value_k<true, T>(F, x) : func_value_k<false, T>(F, x);
}
template <typename T>
__device__ __forceinline__ T func_second_derivative(const pwl_func& F, T x)
{
    return F.kind == PWL_F_SAMPLED ? func_second_derivative_k<true, T>(F, x) : func_second_derivative_k<false, T>(F, x);
}

// FP32 evaluation of f'' (the FP32 design mode) from constants converted
// once per function: a double -> float conversion (or an FP32 division) per
// evaluation would put an operation on the FP64 pipe or several
// instructions in front of every density sample.  Kind-specific constants
// (each formed in FP64, then rounded): Gaussian and Lorentzian
// c = {A, mu, 1/s, A/s^2}; J0(alpha x) c = {A, alpha, -, A alpha^2};
// exponential c = {A, lambda, -, A lambda^2}; polynomial d = the
// coefficients of f'' (k (k-1) p_k at degree k - 2).
struct FuncF {
    int kind;
    float c[4];
    float d[6];
};

__device__ __forceinline__ FuncF make_funcf(const pwl_func& F)
{
    FuncF g{};
    g.kind = F.kind;
    switch (F.kind) {
    case PWL_F_GAUSSIAN:
    case PWL_F_LORENTZIAN:
        g.c[0] = (float)F.p[0];
        g.c[1] = (float)F.p[1];
        g.c[2] = (float)(1.0 / F.p[2]);
        g.c[3] = (float)(F.p[0] / (F.p[2] * F.p[2]));
        break;
    case PWL_F_BESSEL_J0:
    case PWL_F_EXP:
        g.c[0] = (float)F.p[0];
        g.c[1] = (float)F.p[1];
        g.c[3] = (float)(F.p[0] * F.p[1] * F.p[1]);
        break;
    case PWL_F_SAMPLED:  // evaluated from the samples (sampled_second_derivative)
        break;
    default:  // PWL_F_POLY
        for (int k = 2; k < 8; ++k) g.d[k - 2] = (float)((double)(k * (k - 1)) * F.p[k]);
        break;
    }
    return g;
}

__device__ __forceinline__ float func_second_derivative_f(const FuncF& g, float x)
{
    switch (g.kind) {
    case PWL_F_GAUSSIAN: {
        const float u = (x - g.c[1]) * g.c[2];
        return g.c[3] * (u * u - 1.0f) * expf(-0.5f * u * u);
    }
    case PWL_F_LORENTZIAN: {
        const float u = (x - g.c[1]) * g.c[2];
        const float q = 1.0f + u * u;
        return g.c[3] * (6.0f * u * u - 2.0f) / (q * q * q);
    }
    case PWL_F_BESSEL_J0: {
        const float z = g.c[1] * x;
        float b0, b1;
        bessel_j01(z, b0, b1);
        const float r = (fabsf(z) < 1e-4f) ? 0.5f - z * z * 0.0625f : b1 / z;
        return g.c[3] * (r - b0);
    }
    case PWL_F_EXP:
        return g.c[3] * expf(g.c[1] * x);
    default: {
        float s = 0.0f;
        for (int k = 5; k >= 0; --k) s = s * x + g.d[k];
        return s;
    }
    }
}

// host-side descriptor validation
pwl_status validate_func(const pwl_func* f);

// ---------------------------------------------------------------------------
// device table: FP32 knots, the uniform cell index and its records
// ---------------------------------------------------------------------------
// Two cell indexes over [x_0, x_N] serve the kernels; both use uniform
// cells and the cell function below.
//
// 8-byte index (K cells, forward path):
//   - a cell no knot falls in lies inside one interval i; its record is that
//     interval's line {y_c, s_i}, with y_c the line's value at the cell's
//     anchor x_c = fma((float)c, w, a):  v(x) = y_c + (x - x_c) s_i;
//   - a cell holding knot k (the first one, if several) has the record
//     {tag(k), x_k}, tag = quiet NaN with payload k and a flag when more
//     knots share the cell; the side record S[2k + (x >= x_k)] =
//     {v_k, s_k} (left) or {v_k, s_{k+1}} (right) gives v(x) = v_k + (x - x_k) s.
// 16-byte index (K_b cells, used by the backward and texture paths and by the
// forward path for tables whose 8-byte index would not leave room for two
// CTAs per SM): a record belongs to a knot j, {x_j, v_j, s_j, s_{j+1}}
// (forward) or {x_j, j, s_j, s_{j+1}} (backward) with s_j the slope of
// interval j (s_0 := s_1, s_{N+1} := s_N), so that
// v(x) = v_j + (x - x_j) (x <= x_j ? s_j : s_{j+1}) on [x_{j-1}, x_{j+1}];
// a cell holds the record of its first knot or, if no knot falls in it, of
// the last knot before it; when several knots share a cell, the w field is a
// link (quiet NaN whose payload indexes the next knot's record in the chain
// area after the K_b cell records).
constexpr uint32_t kLinkTag = 0x7FC00000u;
constexpr uint32_t kLinkMask = 0x003FFFFFu;
constexpr uint32_t kKnotTagMask = 0x001FFFFFu;  // knot index in a forward knot-cell tag
constexpr uint32_t kKnotTagChain = 0x00200000u; // more knots share the cell
// A backward record of a knot-free cell (the cell lies inside interval j + 1,
// right of knot j) sets bit 31 of its index field and carries 1/h_{j+1} in
// place of s_j: {x_j, j | kInsideFlag, 1/h_{j+1}, s_{j+1}}.
constexpr uint32_t kInsideFlag = 0x80000000u;

__device__ __forceinline__ bool is_link(float w)
{
    return (__float_as_uint(w) & 0xFFC00000u) == kLinkTag;
}
__device__ __forceinline__ int link_index(float w) { return (int)(__float_as_uint(w) & kLinkMask); }
__device__ __forceinline__ float make_link(int j) { return __uint_as_float(kLinkTag | (uint32_t)j); }
__device__ __forceinline__ float make_knot_tag(int k, bool chain)
{
    return __uint_as_float(kLinkTag | (chain ? kKnotTagChain : 0u) | (uint32_t)k);
}

// Cell of a point already clamped to [a, b]: c = trunc(x * inv_w + off)
// with one rounding (fma), clamped to [0, K-1].  Monotone in x, which is
// what makes the record lookup exact; the table builder uses this very
// function on the knots.
__device__ __forceinline__ int cell_of(float xc, float inv_w, float off, int K)
{
    int c = __float2int_rz(__fmaf_rn(xc, inv_w, off));
    return min(max(c, 0), K - 1);
}

// cell_of, and the cell number as a float, without float <-> int
// conversions: for 0 <= t < 2^23, t + 2^23 rounded toward -inf is
// 2^23 + floor(t) (the spacing of floats in [2^23, 2^24) is 1), so floor(t)
// is the float (t + 2^23) - 2^23 and, as an integer, the low mantissa bits
// of its sum with 2^23.  Clamped like cell_of, it returns the same cell for
// every finite t and for NaN (cell 0); needs K <= 2^22.
__device__ __forceinline__ int cell_of_f(float xc, float inv_w, float off, int K, float& cf)
{
    const float t = __fmaf_rn(xc, inv_w, off);
    cf = fminf(fmaxf(__fsub_rn(__fadd_rd(t, 0x1p23f), 0x1p23f), 0.0f), (float)(K - 1));
    return __float_as_int(__fadd_rn(cf, 0x1p23f)) - 0x4B000000;
}

// clamp to [a, b] with NaN propagation
__device__ __forceinline__ float clamp_nan(float x, float a, float b)
{
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(x), "f"(a));
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(r), "f"(b));
    return r;
}

// Device-side status of a table, written by the build kernels and read by
// every kernel that uses the table (so that an asynchronous update needs no
// host round trip).
struct TableHeader {
    int32_t status;      // bit 0: knots not strictly increasing; bit 1: non-finite knot or value;
                         // bit 2: slope or reciprocal length not finite in FP32;
                         // bit 3: an update moved an end knot
    uint32_t hmin_bits;  // shortest interval (positive float, ordered as uint)
    int32_t n_chain_b;   // backward index: chain records after the K_b cell records
    int32_t max_chain_b; // backward index: most chain hops any query can need
    int32_t n_chain_f;   // forward index: knots that share a cell with the previous knot
    int32_t max_chain_f; // forward index: most extra knots in one cell
    int32_t pad[2];
};

}  // namespace pwl

// The opaque handle behind pwl_table.
struct pwl_table_s {
    int device;
    int64_t N;
    int32_t dtype;
    float a, b;
    // forward index
    int64_t K;
    float inv_w, off, w;
    int64_t n_chain_f;
    // backward / texture index
    int64_t Kb;
    float inv_w_b, off_b;
    int64_t n_chain_b;      // at the last synchronous build
    int64_t chain_reserve_b;  // chain records the backward kernel stages in shared memory
    void* buf_base;    // header, knots, values, slopes, build scratch
    void* buf_rec;     // index records
    pwl::TableHeader* hdr;
    float* xk;
    float* vk;
    float* slope;
    float* inv_h;
    void* vstore;      // N+1 values in dtype
    int* cj;           // build scratch: cell of every knot
    int* cpos;         // build scratch: chain slot of every knot
    float2* recP;      // forward, 8-byte layout: K cell records
    float2* recS;      // forward, 8-byte layout: 2 (N+1) side records
    float2* recS8;     // forward, 8-byte layout with one side record per knot: N+1 records {v_k, s_{k+1}}
    float4* rec16;     // forward, 16-byte layout on the K_b grid: K_b + N + 1 records
    float4* rec_b;     // backward: K_b + N + 1 records
    int32_t layout;    // forward layout pwl_eval uses: 0 = 8-byte cells, 1 = 16-byte cells,
                       // 2 = 8-byte cells with one side record per knot
    cudaArray_t tex_array;
    cudaTextureObject_t tex;
};
