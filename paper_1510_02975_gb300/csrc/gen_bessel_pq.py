"""Writes pwl_bessel_tables.cuh: Chebyshev coefficients of the modulus-phase
functions of J0 and J1 for x >= 8.

For nu = 0, 1 (DLMF 10.17.3-4 and the definitions of P_nu, Q_nu there):
    J_nu(x) = sqrt(2 / (pi x)) (P_nu(x) cos chi - Q_nu(x) sin chi),
    Y_nu(x) = sqrt(2 / (pi x)) (P_nu(x) sin chi + Q_nu(x) cos chi),
    chi = x - (2 nu + 1) pi / 4,
so that P_nu = sqrt(pi x / 2) (J_nu cos chi + Y_nu sin chi) and
Q_nu = sqrt(pi x / 2) (Y_nu cos chi - J_nu sin chi).  Both are smooth in
u = (8 / x)^2 on (0, 1] (P_nu -> 1, Q_nu ~ (4 nu^2 - 1) / (8 x)).  This
script evaluates P_nu and (x / 8) Q_nu with mpmath at 45 digits at the n
Chebyshev nodes of w = 2 u - 1 and prints the Chebyshev interpolation
coefficients (the truncated series is accurate to ~1e-19 at n = 16).

Run: python gen_bessel_pq.py > pwl_bessel_tables.cuh   (needs mpmath)
"""
import mpmath as mp

N_COEF = 16


def pq(nu, x):
    chi = x - (2 * nu + 1) * mp.pi / 4
    s = mp.sqrt(mp.pi * x / 2)
    j, y = mp.besselj(nu, x), mp.bessely(nu, x)
    return s * (j * mp.cos(chi) + y * mp.sin(chi)), s * (y * mp.cos(chi) - j * mp.sin(chi))


def chebyshev(nu, which, n):
    vals = []
    for k in range(n):
        w = mp.cos(mp.pi * (k + mp.mpf(1) / 2) / n)
        u = (w + 1) / 2
        x = 8 / mp.sqrt(u)
        p, q = pq(nu, x)
        vals.append(p if which == "P" else q * x / 8)
    out = []
    for j in range(n):
        s = mp.fsum(vals[k] * mp.cos(mp.pi * j * (k + mp.mpf(1) / 2) / n) for k in range(n))
        out.append(s * (1 if j == 0 else 2) / n)
    return out


def main():
    mp.mp.dps = 45
    print("// pwl_bessel_tables.cuh -- written by gen_bessel_pq.py; do not edit.")
    print("// Chebyshev coefficients c_j, j = 0..%d, in w = 2 (8/x)^2 - 1 (x >= 8) of" % (N_COEF - 1))
    print("// P_nu(x) and (x/8) Q_nu(x), the modulus-phase functions of J0 and J1.")
    print("#pragma once")
    print("namespace pwl {")
    coef = {(nu, which): chebyshev(nu, which, N_COEF) for nu in (0, 1) for which in ("P", "Q")}
    for (nu, which), c in coef.items():
        body = ",\n    ".join(mp.nstr(v, 20, min_fixed=1, max_fixed=0) for v in c)
        print("static __device__ __constant__ double kBessel%s%d[%d] = {\n    %s};" % (which, nu, N_COEF, body))
    print("}  // namespace pwl")


if __name__ == "__main__":
    main()
