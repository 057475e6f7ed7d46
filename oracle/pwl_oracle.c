/*
 * pwl_oracle.c -- plain FP64 CPU oracle for the continuous piecewise-linear
 * (CPWL) approximation method of Berjon, Gallego, Cuevas, Moran and Garcia,
 * "Optimal Piecewise Linear Function Approximation for GPU-based
 * Applications" (IEEE Trans. Cybernetics, 2015).
 *
 * TEST INFRASTRUCTURE.  This file is the slow, obviously correct reference
 * that the CUDA library is checked against.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Everything is FP64 and written in the order and notation of the paper:
 *   - f and f'' of the analytic test functions            (Sections V-VI)
 *   - local knot density |f''|^{2/5}                       (Eq. 16)
 *   - cumulative knot distribution F                       (Eq. 18)
 *   - knots with F(x_i) = i/N, x_0 = a, x_N = b             (Eq. 17)
 *   - interpolant values f(x_i)                            (Eq. 3)
 *   - L2 projection: Gram system M c = b, Thomas algorithm (Eqs. 4-6)
 *   - CPWL evaluation                                      (Algorithm 1)
 *   - gradients of Algorithm 1 w.r.t. x, v(x_i), x_i        (calculus on Eq. 8)
 *   - L2 distances for the error results                   (Results 1-6)
 *   - the direct evaluations the paper compares against    (Section V)
 *
 * Readings of points the paper leaves open (each listed in the design notes):
 *   - the density uses |f''| (Eq. 16 has the absolute value, Eq. 18 drops it);
 *   - F is integrated with the midpoint rule on M uniform cells;
 *   - a knot is never placed inside a run of zero-density cells: for target
 *     tau the cell is the largest k with G_k <= tau and d_k > 0;
 *   - if the integral of |f''|^{2/5} is zero (f linear) the partition is
 *     uniform and the call returns 1;
 *   - Algorithm 1 is extended to x = x_N (interval N, delta = 1) and clamps x
 *     outside [a, b]; a NaN query gives NaN;
 *   - <f, phi_i> uses Q-point Gauss-Legendre quadrature per interval.
 */
#define _DEFAULT_SOURCE 1 /* j0, j1, M_PI */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Analytic test functions.  p[] meaning per kind:
 *   GAUSSIAN   : A exp(-(x-mu)^2 / (2 s^2))       p = {A, mu, s}
 *   LORENTZIAN : A / (1 + ((x-x0)/g)^2)            p = {A, x0, g}
 *   BESSEL_J0  : A J0(alpha x)                     p = {A, alpha}
 *   POLY       : sum_{k<=7} p[k] x^k
 *   EXP        : A exp(lambda x)                   p = {A, lambda}
 *   SAMPLED    : S = p[0] samples f(a + j h), h = (b-a)/(S-1), j < S, at the
 *                host address whose 64 bits p[1] holds                      */
typedef struct {
    int32_t kind;
    int32_t pad;
    double a, b;
    double p[8];
} orc_func;

enum { ORC_GAUSSIAN = 0, ORC_LORENTZIAN = 1, ORC_BESSEL_J0 = 2, ORC_POLY = 3, ORC_EXP = 4, ORC_SAMPLED = 5 };

/* A sampled f: the samples and the cell of x.  With u = (x - a)/h the cell
 * is j = floor(u) kept in [1, S-3], so that samples j-1 .. j+2 exist; t =
 * u - j (outside [0, 1) only in the two end cells). */
static const double* orc_samples(const orc_func* F)
{
    uint64_t addr;
    memcpy(&addr, &F->p[1], sizeof(addr));
    return (const double*)(uintptr_t)addr;
}

static int64_t orc_sample_cell(const orc_func* F, double x, double* t)
{
    int64_t S = (int64_t)F->p[0];
    double h = (F->b - F->a) / (double)(S - 1);
    double u = (x - F->a) / h;
    int64_t j = (int64_t)floor(u);
    if (j < 1) j = 1;
    if (j > S - 3) j = S - 3;
    *t = u - (double)j;
    return j;
}

/* f: Lagrange's form of the cubic through (m, s_{j+m}), m = -1, 0, 1, 2 */
static double orc_sampled_f(const orc_func* F, double x)
{
    double t;
    int64_t j = orc_sample_cell(F, x, &t);
    const double* s = orc_samples(F);
    double y = 0.0;
    for (int m = -1; m <= 2; ++m) {
        double w = 1.0;
        for (int k = -1; k <= 2; ++k)
            if (k != m) w *= (t - (double)k) / (double)(m - k);
        y += w * s[j + m];
    }
    return y;
}

/* f'': the second differences D_i = (s_{i-1} - 2 s_i + s_{i+1}) / h^2 at
 * samples j and j+1, joined by a straight line */
static double orc_sampled_f2(const orc_func* F, double x)
{
    double t;
    int64_t j = orc_sample_cell(F, x, &t);
    const double* s = orc_samples(F);
    double h = (F->b - F->a) / (F->p[0] - 1.0);
    double Dj = (s[j - 1] - 2.0 * s[j] + s[j + 1]) / (h * h);
    double Dk = (s[j] - 2.0 * s[j + 1] + s[j + 2]) / (h * h);
    return (1.0 - t) * Dj + t * Dk;
}

/* ------------------------------------------------------------------------ */
/* f and f''                                                                 */
/* ------------------------------------------------------------------------ */

double orc_f(const orc_func* F, double x)
{
    switch (F->kind) {
    case ORC_GAUSSIAN: {
        double u = (x - F->p[1]) / F->p[2];
        return F->p[0] * exp(-0.5 * u * u);
    }
    case ORC_LORENTZIAN: {
        double u = (x - F->p[1]) / F->p[2];
        return F->p[0] / (1.0 + u * u);
    }
    case ORC_BESSEL_J0:
        return F->p[0] * j0(F->p[1] * x);
    case ORC_POLY: {
        double s = 0.0;
        for (int k = 7; k >= 0; --k) s = s * x + F->p[k];
        return s;
    }
    case ORC_EXP:
        return F->p[0] * exp(F->p[1] * x);
    case ORC_SAMPLED:
        return orc_sampled_f(F, x);
    }
    return NAN;
}

/* Second derivative, written out for each kind:
 *   Gaussian   : A (u^2 - 1) / s^2 * exp(-u^2/2),        u = (x-mu)/s
 *   Lorentzian : A (6u^2 - 2) / (g^2 (1+u^2)^3),         u = (x-x0)/g
 *   J0(alpha x): A alpha^2 (J1(z)/z - J0(z)),            z = alpha x
 *                (Bessel's equation z^2 J0'' + z J0' + z^2 J0 = 0, J0' = -J1;
 *                 J1(z)/z -> 1/2 as z -> 0)
 *   poly       : sum k (k-1) p_k x^(k-2)
 *   exp        : A lambda^2 exp(lambda x)                                 */
/* f at n points (the reference of the direct-evaluation comparisons). */
void orc_f_many(const orc_func* F, const double* x, int64_t n, double* out)
{
    for (int64_t q = 0; q < n; ++q) out[q] = orc_f(F, x[q]);
}

/* The first term of the asymptotic expansion of J0 for large argument that
 * the paper times as a fast alternative to J0 (Section V-C):
 *     A J0(z) ~ A sqrt(2 / (pi z)) cos(z - pi/4),  z = alpha x,
 * evaluated as written (z > 0; the expression is the definition, its error
 * against J0 is that of the truncated expansion). */
void orc_j0_one_term(const orc_func* F, const double* x, int64_t n, double* out)
{
    for (int64_t q = 0; q < n; ++q) {
        const double z = F->p[1] * x[q];
        out[q] = F->p[0] * sqrt(2.0 / (M_PI * z)) * cos(z - M_PI / 4.0);
    }
}

double orc_f2(const orc_func* F, double x)
{
    switch (F->kind) {
    case ORC_GAUSSIAN: {
        double s = F->p[2];
        double u = (x - F->p[1]) / s;
        return F->p[0] * (u * u - 1.0) / (s * s) * exp(-0.5 * u * u);
    }
    case ORC_LORENTZIAN: {
        double g = F->p[2];
        double u = (x - F->p[1]) / g;
        double q = 1.0 + u * u;
        return F->p[0] * (6.0 * u * u - 2.0) / (g * g * q * q * q);
    }
    case ORC_BESSEL_J0: {
        double al = F->p[1];
        double z = al * x;
        double j1_over_z = (fabs(z) < 1e-8) ? 0.5 - z * z / 16.0 : j1(z) / z;
        return F->p[0] * al * al * (j1_over_z - j0(z));
    }
    case ORC_POLY: {
        double s = 0.0;
        for (int k = 7; k >= 2; --k) s = s * x + (double)(k * (k - 1)) * F->p[k];
        return s;
    }
    case ORC_EXP:
        return F->p[0] * F->p[1] * F->p[1] * exp(F->p[1] * x);
    case ORC_SAMPLED:
        return orc_sampled_f2(F, x);
    }
    return NAN;
}

/* ------------------------------------------------------------------------ */
/* Design: knot placement by equidistribution (Section III-B)                */
/* ------------------------------------------------------------------------ */

/* Local knot density (Eq. 16) sampled at the midpoints of M uniform cells:
 *   d_k = |f''(t_k)|^{2/5},  t_k = a + (k + 1/2) (b - a) / M,  k < M.        */
void orc_density(const orc_func* F, int64_t M, double* d)
{
    double delta = (F->b - F->a) / (double)M;
    for (int64_t k = 0; k < M; ++k) {
        double t = F->a + ((double)k + 0.5) * delta;
        d[k] = pow(fabs(orc_f2(F, t)), 0.4);
    }
}

/* Unnormalised cumulative distribution (numerator of Eq. 18) by the midpoint
 * rule: G_0 = 0, G_k = delta * sum_{j<k} d_j, k = 0..M.  The running sum is
 * compensated (Neumaier) so that every G_k is the correctly rounded value of
 * the exact sum up to a few ulp.                                            */
void orc_cumulative(const double* d, int64_t M, double delta, double* G)
{
    double s = 0.0, c = 0.0;
    G[0] = 0.0;
    for (int64_t k = 0; k < M; ++k) {
        double t = s + d[k];
        if (fabs(s) >= fabs(d[k])) c += (s - t) + d[k];
        else c += (d[k] - t) + s;
        s = t;
        G[k + 1] = delta * (s + c);
    }
}

/* Knots of the partition T* (Eq. 17): x_0 = a, x_N = b and, for 0 < i < N,
 * x_i solves F(x_i) = i/N.  With tau_i = i G_M / N, the cell is the largest k
 * with G_k <= tau_i and d_k > 0, and inside it F is linear, so
 *   x_i = a + k delta + (tau_i - G_k) / d_k.
 * Returns 0, or 1 when G_M == 0 (the uniform partition is returned).        */
int orc_invert(const double* d, const double* G, int64_t M, double a, double b,
               int64_t N, double* knots)
{
    double delta = (b - a) / (double)M;
    double GM = G[M];
    knots[0] = a;
    knots[N] = b;
    if (!(GM > 0.0)) {
        for (int64_t i = 1; i < N; ++i) knots[i] = a + (double)i * (b - a) / (double)N;
        return 1;
    }
    for (int64_t i = 1; i < N; ++i) {
        double tau = (double)i * GM / (double)N;
        /* largest k in [0, M-1] with G_k <= tau (binary search) */
        int64_t lo = 0, hi = M - 1;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo + 1) / 2;
            if (G[mid] <= tau) lo = mid; else hi = mid - 1;
        }
        int64_t k = lo;
        while (k > 0 && !(d[k] > 0.0)) --k;
        double x = a + (double)k * delta;
        if (d[k] > 0.0) {
            double step = (tau - G[k]) / d[k];
            if (step < 0.0) step = 0.0;
            if (step > delta) step = delta;
            x += step;
        }
        knots[i] = x;
    }
    return 0;
}

/* The whole design step: density -> cumulative -> inversion.  G (M+1) and
 * d (M) are returned for inspection when the pointers are non-NULL.         */
int orc_design(const orc_func* F, int64_t N, int64_t M, double* knots, double* d_out,
               double* G_out)
{
    double* d = d_out ? d_out : (double*)malloc(sizeof(double) * (size_t)M);
    double* G = G_out ? G_out : (double*)malloc(sizeof(double) * (size_t)(M + 1));
    orc_density(F, M, d);
    orc_cumulative(d, M, (F->b - F->a) / (double)M, G);
    int rc = orc_invert(d, G, M, F->a, F->b, N, knots);
    if (!d_out) free(d);
    if (!G_out) free(G);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Vertex values: interpolant pi_T (Eq. 3) and projection P_T (Eqs. 4-6)     */
/* ------------------------------------------------------------------------ */

void orc_interp_values(const orc_func* F, const double* knots, int64_t N, double* v)
{
    for (int64_t i = 0; i <= N; ++i) v[i] = orc_f(F, knots[i]);
}

/* Q-point Gauss-Legendre rule on [-1, 1]: the nodes are the roots of the
 * Legendre polynomial P_Q, found by Newton's method from the asymptotic guess
 * cos(pi (i - 1/4) / (Q + 1/2)); P_Q and P_Q' come from the three-term
 * recurrence (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1} and
 * (x^2 - 1) P_Q' = Q (x P_Q - P_{Q-1}); weights 2 / ((1 - x^2) P_Q'(x)^2).
 * Nodes are returned in increasing order.                                   */
void orc_gauss_legendre(int Q, double* nodes, double* weights)
{
    for (int i = 1; i <= Q; ++i) {
        double x = cos(M_PI * ((double)i - 0.25) / ((double)Q + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int n = 1; n < Q; ++n) {
                double p2 = ((2.0 * n + 1.0) * x * p1 - (double)n * p0) / (double)(n + 1);
                p0 = p1;
                p1 = p2;
            }
            /* now p1 = P_Q(x), p0 = P_{Q-1}(x) */
            dp = (double)Q * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int n = 1; n < Q; ++n) {
                double p2 = ((2.0 * n + 1.0) * x * p1 - (double)n * p0) / (double)(n + 1);
                p0 = p1;
                p1 = p2;
            }
            dp = (double)Q * (x * p1 - p0) / (x * x - 1.0);
        }
        nodes[Q - i] = x; /* cos is decreasing in i: store ascending */
        weights[Q - i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

/* Load vector b_i = <f, phi_i> (Eq. 4 with the hat functions of Eq. 1), by
 * Q-point Gauss-Legendre quadrature on every interval I_j = [x_{j-1}, x_j]:
 * on I_j only phi_{j-1} = (x_j - t)/h_j and phi_j = (t - x_{j-1})/h_j are
 * non-zero.  At the node t = mid + (h_j/2) xi_q these are exactly
 * (1 - xi_q)/2 and (1 + xi_q)/2; the oracle uses those values, because
 * forming x_j - t in floating point cancels (it loses about |x|/h_j ulps
 * when the knots are far from 0 compared with h_j).                         */
void orc_load_vector(const orc_func* F, const double* knots, int64_t N, int Q, double* bvec)
{
    double xi[64], w[64];
    orc_gauss_legendre(Q, xi, w);
    for (int64_t i = 0; i <= N; ++i) bvec[i] = 0.0;
    for (int64_t j = 1; j <= N; ++j) {
        double xl = knots[j - 1], xr = knots[j];
        double h = xr - xl;
        double mid = 0.5 * (xl + xr), half = 0.5 * h;
        for (int q = 0; q < Q; ++q) {
            double t = mid + half * xi[q];
            double fw = half * w[q] * orc_f(F, t);
            bvec[j - 1] += fw * ((1.0 - xi[q]) * 0.5);
            bvec[j] += fw * ((1.0 + xi[q]) * 0.5);
        }
    }
}

/* Gram matrix M = (<phi_i, phi_j>) of the hat basis (Section II-B): it is
 * tridiagonal with, per interval of length h, the 2x2 block
 * [[h/3, h/6], [h/6, h/3]] (the integral of (h/3)(D0^2 + D1^2 + D0 D1) form
 * used in the proof of Result 2).  lower[i] = M_{i,i-1}, diag[i] = M_{i,i},
 * upper[i] = M_{i,i+1}.                                                     */
void orc_gram(const double* knots, int64_t N, double* lower, double* diag, double* upper)
{
    for (int64_t i = 0; i <= N; ++i) {
        double hl = (i > 0) ? knots[i] - knots[i - 1] : 0.0;
        double hr = (i < N) ? knots[i + 1] - knots[i] : 0.0;
        lower[i] = hl / 6.0;
        diag[i] = (hl + hr) / 3.0;
        upper[i] = hr / 6.0;
    }
}

/* Thomas algorithm (Gaussian elimination without pivoting on a tridiagonal
 * system), which the paper names for M c = b.  lower[0] and upper[n-1] are
 * ignored.  Solution overwrites rhs.                                        */
void orc_thomas(int64_t n, const double* lower, const double* diag, const double* upper,
                double* rhs)
{
    double* cp = (double*)malloc(sizeof(double) * (size_t)n);
    double denom = diag[0];
    cp[0] = (n > 1) ? upper[0] / denom : 0.0;
    rhs[0] = rhs[0] / denom;
    for (int64_t i = 1; i < n; ++i) {
        denom = diag[i] - lower[i] * cp[i - 1];
        cp[i] = (i < n - 1) ? upper[i] / denom : 0.0;
        rhs[i] = (rhs[i] - lower[i] * rhs[i - 1]) / denom;
    }
    for (int64_t i = n - 2; i >= 0; --i) rhs[i] -= cp[i] * rhs[i + 1];
    free(cp);
}

/* P_T f vertex values c_i (Eq. 6): assemble M and b, solve M c = b.         */
void orc_project_values(const orc_func* F, const double* knots, int64_t N, int Q, double* c)
{
    int64_t n = N + 1;
    double* lo = (double*)malloc(sizeof(double) * (size_t)n);
    double* di = (double*)malloc(sizeof(double) * (size_t)n);
    double* up = (double*)malloc(sizeof(double) * (size_t)n);
    orc_gram(knots, N, lo, di, up);
    orc_load_vector(F, knots, N, Q, c);
    orc_thomas(n, lo, di, up, c);
    free(lo);
    free(di);
    free(up);
}

/* ------------------------------------------------------------------------ */
/* Evaluation (Algorithm 1) and its gradients                                */
/* ------------------------------------------------------------------------ */

/* Index i in [1, N] of the interval holding x (already in [x_0, x_N]):
 * the first knot strictly greater than x, i.e. x_{i-1} <= x < x_i, found by
 * binary search (upper bound); x = x_N maps to i = N.                       */
static int64_t orc_interval(const double* xk, int64_t N, double x)
{
    int64_t lo = 0, hi = N + 1; /* first index with xk[idx] > x, in [0, N+1] */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (xk[mid] > x) hi = mid; else lo = mid + 1;
    }
    int64_t i = lo;
    if (i < 1) i = 1;
    if (i > N) i = N;
    return i;
}

/* Algorithm 1: locate i with x_{i-1} <= x < x_i, delta = (x - x_{i-1}) /
 * (x_i - x_{i-1}), return (1 - delta) v_{i-1} + delta v_i.  x is clamped to
 * [x_0, x_N]; NaN stays NaN.                                                 */
void orc_eval(const double* xk, const double* vk, int64_t N, const double* x, double* y,
              int64_t m)
{
    for (int64_t q = 0; q < m; ++q) {
        double xq = x[q];
        if (isnan(xq)) { y[q] = xq; continue; }
        if (xq < xk[0]) xq = xk[0];
        if (xq > xk[N]) xq = xk[N];
        int64_t i = orc_interval(xk, N, xq);
        double delta = (xq - xk[i - 1]) / (xk[i] - xk[i - 1]);
        y[q] = (1.0 - delta) * vk[i - 1] + delta * vk[i];
    }
}

/* Gradients of Algorithm 1 for upstream gradients gy[q].  With
 * h = x_i - x_{i-1}, delta = (x - x_{i-1})/h and s = (v_i - v_{i-1})/h:
 *   dy/dx       = s
 *   dy/dv_{i-1} = 1 - delta,       dy/dv_i = delta
 *   dy/dx_{i-1} = -s (1 - delta),  dy/dx_i = -s delta.
 * A clamped query (x < x_0 or x > x_N) has y = v_0 (or v_N): dy/dx = 0 and
 * only that vertex gets gy.  NaN queries give gx = NaN and no table terms.
 * gv and gxk are accumulated (+=).  If gv_abs / gxk_abs are non-NULL they
 * receive the sums of the absolute values of the same terms.                */
void orc_eval_grad(const double* xk, const double* vk, int64_t N, const double* x,
                   const double* gy, int64_t m, double* gx, double* gv, double* gxk,
                   double* gv_abs, double* gxk_abs)
{
    for (int64_t q = 0; q < m; ++q) {
        double xq = x[q], g = gy[q];
        if (isnan(xq)) { gx[q] = xq; continue; }
        if (xq < xk[0] || xq > xk[N]) {
            int64_t e = (xq < xk[0]) ? 0 : N;
            gx[q] = 0.0;
            gv[e] += g;
            if (gv_abs) gv_abs[e] += fabs(g);
            continue;
        }
        int64_t i = orc_interval(xk, N, xq);
        double h = xk[i] - xk[i - 1];
        double delta = (xq - xk[i - 1]) / h;
        double s = (vk[i] - vk[i - 1]) / h;
        gx[q] = g * s;
        gv[i - 1] += g * (1.0 - delta);
        gv[i] += g * delta;
        gxk[i - 1] += -g * s * (1.0 - delta);
        gxk[i] += -g * s * delta;
        if (gv_abs) {
            gv_abs[i - 1] += fabs(g * (1.0 - delta));
            gv_abs[i] += fabs(g * delta);
        }
        if (gxk_abs) {
            gxk_abs[i - 1] += fabs(g * s * (1.0 - delta));
            gxk_abs[i] += fabs(g * s * delta);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Error measures for Results 1-6                                            */
/* ------------------------------------------------------------------------ */

/* L2 distance ||f - v|| on [x_0, x_N] (the norm induced by Eq. 4) for the
 * CPWL v with knots xk and values vk: every interval is split into `sub`
 * equal parts, each integrated with Q-point Gauss-Legendre.  If per_interval
 * is non-NULL it receives the squared error on each interval (index 1..N;
 * entry 0 is set to 0).                                                     */
double orc_l2_error(const orc_func* F, const double* xk, const double* vk, int64_t N, int Q,
                    int sub, double* per_interval)
{
    double xi[64], w[64];
    orc_gauss_legendre(Q, xi, w);
    double total = 0.0;
    if (per_interval) per_interval[0] = 0.0;
    for (int64_t j = 1; j <= N; ++j) {
        double xl = xk[j - 1], xr = xk[j], h = xr - xl;
        double acc = 0.0;
        for (int s = 0; s < sub; ++s) {
            double l = xl + h * (double)s / (double)sub;
            double r = xl + h * (double)(s + 1) / (double)sub;
            double mid = 0.5 * (l + r), half = 0.5 * (r - l);
            for (int q = 0; q < Q; ++q) {
                double t = mid + half * xi[q];
                double delta = (t - xl) / h;
                double v = (1.0 - delta) * vk[j - 1] + delta * vk[j];
                double e = orc_f(F, t) - v;
                acc += half * w[q] * e * e;
            }
        }
        if (per_interval) per_interval[j] = acc;
        total += acc;
    }
    return sqrt(total);
}

/* Integral over [a, b] of |f''|^p (p = 2/5 gives the constant in Result 4,
 * p = 2 gives ||f''||^2 in Result 6), by `n` equal sub-intervals of Q-point
 * Gauss-Legendre.                                                           */
double orc_integral_abs_f2_pow(const orc_func* F, double p, int64_t n, int Q)
{
    double xi[64], w[64];
    orc_gauss_legendre(Q, xi, w);
    double a = F->a, b = F->b, acc = 0.0;
    for (int64_t s = 0; s < n; ++s) {
        double l = a + (b - a) * (double)s / (double)n;
        double r = a + (b - a) * (double)(s + 1) / (double)n;
        double mid = 0.5 * (l + r), half = 0.5 * (r - l);
        for (int q = 0; q < Q; ++q) {
            double t = mid + half * xi[q];
            acc += half * w[q] * pow(fabs(orc_f2(F, t)), p);
        }
    }
    return acc;
}
