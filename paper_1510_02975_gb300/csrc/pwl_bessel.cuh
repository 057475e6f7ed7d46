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
// absolute error ~3e-16.
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
    return (p * (c + s) - q * (s - c)) * rsqrt(3.14159265358979323846 * ax);
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
    const double r = (p * (s - c) + q * (s + c)) * rsqrt(3.14159265358979323846 * ax);
    return x < 0.0 ? -r : r;
}

// FP32 (the FP32 design mode): the library's j0f / j1f (absolute error
// ~5e-7), within the FP32 mode's knot bound.
__device__ __forceinline__ float bessel_j0(float x) { return j0f(x); }
__device__ __forceinline__ float bessel_j1(float x) { return j1f(x); }

// J0 and J1 at the same point (f'' needs both): one sincos and one square
// root for the two.
__device__ __forceinline__ void bessel_j01(double x, double& j0v, double& j1v)
{
    const double ax = fabs(x);
    if (ax < 8.0) {
        j0v = j0(x);
        j1v = j1(x);
        return;
    }
    const double t = 8.0 / ax, w = 2.0 * t * t - 1.0;
    const double p0 = chebyshev_sum<double, 16>(kBesselP0, w), q0 = t * chebyshev_sum<double, 16>(kBesselQ0, w);
    const double p1 = chebyshev_sum<double, 16>(kBesselP1, w), q1 = t * chebyshev_sum<double, 16>(kBesselQ1, w);
    double s, c;
    sincos(ax, &s, &c);
    const double r = rsqrt(3.14159265358979323846 * ax);
    j0v = (p0 * (c + s) - q0 * (s - c)) * r;
    const double j1a = (p1 * (s - c) + q1 * (s + c)) * r;
    j1v = x < 0.0 ? -j1a : j1a;
}

__device__ __forceinline__ void bessel_j01(float x, float& j0v, float& j1v)
{
    j0v = j0f(x);
    j1v = j1f(x);
}

}  // namespace pwl
