// pwl_bessel.cuh -- J0 and J1 for the Bessel test function f = A J0(alpha x)
// (Section V) and its second derivative A alpha^2 (J1(z)/z - J0(z)).
//
// Below x = 8 the CUDA library functions are used (their absolute error
// there is ~5e-16 in FP64).  From x = 8 on, the library's FP64 error grows
// to ~1e-13 (J0) and ~4e-13 (J1) by x = 250, which the density |f''|^{2/5}
// turns into knot errors above 1e-12 (b - a) for J0(alpha x) with
// alpha >= 3 on [0, 50].  There the modulus-phase form (DLMF 10.17)
//     J_nu(x) = sqrt(2 / (pi x)) (P_nu(x) cos chi - Q_nu(x) sin chi),
//     chi = x - (2 nu + 1) pi / 4,
// is evaluated with Chebyshev series of P_nu and (x/8) Q_nu in
// w = 2 (8/x)^2 - 1 (pwl_bessel_tables.cuh, from gen_bessel_pq.py), and with
//     cos chi0 = (cos x + sin x) / sqrt 2,   sin chi0 = (sin x - cos x) / sqrt 2,
//     cos chi1 = (sin x - cos x) / sqrt 2,   sin chi1 = -(sin x + cos x) / sqrt 2:
// absolute error ~3e-16 in FP64, and a few FP32 ulps of sqrt(2 / (pi x)) in
// FP32 (the series cut to 6 terms).
#pragma once

#include <math.h>

#include "pwl_bessel_tables.cuh"

namespace pwl {

// Clenshaw sum of c_0 T_0(w) + ... + c_{N-1} T_{N-1}(w)
template <typename T, int N>
__device__ __forceinline__ T chebyshev_sum(const T* c, T w)
{
    T b1 = T(0), b2 = T(0);
#pragma unroll
    for (int j = N - 1; j >= 1; --j) {
        const T b0 = T(2) * w * b1 - b2 + c[j];
        b2 = b1;
        b1 = b0;
    }
    return w * b1 - b2 + c[0];
}

__device__ __forceinline__ double bessel_j0(double x)
{
    const double ax = fabs(x);
    if (ax < 8.0) return j0(x);
    const double t = 8.0 / ax, w = 2.0 * t * t - 1.0;
    const double p = chebyshev_sum<double, 16>(kBesselP0, w);
    const double q = t * chebyshev_sum<double, 16>(kBesselQ0, w);
    double s, c;
    sincos(ax, &s, &c);
    return (p * (c + s) - q * (s - c)) / sqrt(3.14159265358979323846 * ax);
}

__device__ __forceinline__ double bessel_j1(double x)
{
    const double ax = fabs(x);
    if (ax < 8.0) return j1(x);
    const double t = 8.0 / ax, w = 2.0 * t * t - 1.0;
    const double p = chebyshev_sum<double, 16>(kBesselP1, w);
    const double q = t * chebyshev_sum<double, 16>(kBesselQ1, w);
    double s, c;
    sincos(ax, &s, &c);
    const double r = (p * (s - c) + q * (s + c)) / sqrt(3.14159265358979323846 * ax);
    return x < 0.0 ? -r : r;
}

__device__ __forceinline__ float bessel_j0(float x)
{
    const float ax = fabsf(x);
    if (ax < 8.0f) return j0f(x);
    const float t = 8.0f / ax, w = 2.0f * t * t - 1.0f;
    const float p = chebyshev_sum<float, 6>(kBesselP0f, w);
    const float q = t * chebyshev_sum<float, 6>(kBesselQ0f, w);
    float s, c;
    sincosf(ax, &s, &c);
    return (p * (c + s) - q * (s - c)) / sqrtf(3.14159265f * ax);
}

__device__ __forceinline__ float bessel_j1(float x)
{
    const float ax = fabsf(x);
    if (ax < 8.0f) return j1f(x);
    const float t = 8.0f / ax, w = 2.0f * t * t - 1.0f;
    const float p = chebyshev_sum<float, 6>(kBesselP1f, w);
    const float q = t * chebyshev_sum<float, 6>(kBesselQ1f, w);
    float s, c;
    sincosf(ax, &s, &c);
    const float r = (p * (s - c) + q * (s + c)) / sqrtf(3.14159265f * ax);
    return x < 0.0f ? -r : r;
}

}  // namespace pwl
