/*
 * pwl.h -- C ABI of libpwl, a single-GPU (GB300, sm_103a) library that
 * evaluates a continuous function f at very many points through its nearly
 * optimal continuous piecewise-linear (CPWL) approximation, following
 * Berjon et al., "Optimal Piecewise Linear Function Approximation for
 * GPU-based Applications" (IEEE Trans. Cybernetics, 2015).
 *
 * The calls follow the paper's statement of the problem (Section II-B): f is
 * continuous on I = [a, b]; a partition T = {a = x_0 < ... < x_N = b} has N
 * intervals and N+1 knots; a CPWL function v is given by its nodal values
 * v(x_0..x_N) (Eq. 2); Algorithm 1 evaluates v at a point x*.
 *
 * Conventions shared by every call:
 *   - Pointers named d_* (and every array argument unless marked "host") are
 *     device pointers owned by the caller.  The library owns only the opaque
 *     handles it returns (pwl_table, pwl_batch, pwl_channels), freed by the
 *     matching *_destroy call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work on it and return without waiting, except
 *     where a call says "synchronizes".
 *   - Every call returns a pwl_status.  Arguments are validated on the host
 *     before anything is launched; on failure nothing is enqueued and
 *     pwl_last_error() describes the problem (thread-local string).
 *     PWL_ECUDA reports a CUDA launch or runtime error.
 *   - Workspace arguments: scratch device memory of at least the size the
 *     matching *_workspace_size call returns, 256-byte aligned, not used by
 *     another call that runs at the same time.
 *   - Sizes: 1 <= N <= 1048575 intervals per function; m >= 0 queries
 *     (m == 0 is a no-op).
 */
#ifndef PWL_H
#define PWL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PWL_OK = 0,
    PWL_EINVAL = 1,   /* bad argument (size, pointer, non-increasing knots, ...) */
    PWL_ENOMEM = 2,   /* device or host allocation failed                         */
    PWL_ECUDA = 3,    /* CUDA runtime / launch error                             */
    PWL_ENOTSUP = 4,  /* combination not supported                               */
    PWL_ETIMEOUT = 5  /* a bounded device loop hit its iteration cap             */
} pwl_status;

/* Analytic functions f on [a, b] with their second derivative in closed form
 * (the design step needs f'').  Parameters p[]:
 *   PWL_F_GAUSSIAN   A exp(-(x - mu)^2 / (2 s^2))     p = {A, mu, s}     (Section V-A)
 *   PWL_F_LORENTZIAN A / (1 + ((x - x0) / g)^2)        p = {A, x0, g}     (Eq. 25 with
 *                    A = 1/(pi g) gives the paper's normalised form, Section V-B)
 *   PWL_F_BESSEL_J0  A J0(alpha x)                     p = {A, alpha}     (Section V-C)
 *   PWL_F_POLY       sum_{k=0..7} p[k] x^k                               (Fig. 1's quintic)
 *   PWL_F_EXP        A exp(lambda x)                   p = {A, lambda}
 * and a function given by samples (any continuous f the caller can tabulate):
 *   PWL_F_SAMPLED    S >= 4 FP64 samples s_j = f(a + j h), h = (b - a)/(S - 1),
 *                    j = 0..S-1, in device memory that the caller keeps alive
 *                    while calls use the descriptor; p[0] = S, p[1] holds
 *                    the 64 bits of the device address, p[2..4] = h, 1/h,
 *                    1/h^2 (pwl_func_sampled writes them all).  With
 *                    u = (x - a) (1/h) and
 *                    j = min(max(floor(u), 1), S - 3):
 *                      f(x)   = the cubic through samples j-1 .. j+2 at u;
 *                      f''(x) = D_j + (u - j)(D_{j+1} - D_j), the linear
 *                               interpolant (extrapolant in the end cells) of
 *                               the second differences
 *                               D_j = (s_{j-1} - 2 s_j + s_{j+1}) / h^2.
 *                    Both are exact when f is a polynomial of degree <= 3.   */
typedef enum {
    PWL_F_GAUSSIAN = 0,
    PWL_F_LORENTZIAN = 1,
    PWL_F_BESSEL_J0 = 2,
    PWL_F_POLY = 3,
    PWL_F_EXP = 4,
    PWL_F_SAMPLED = 5
} pwl_kind;

typedef struct {
    int32_t kind;     /* pwl_kind */
    int32_t reserved; /* must be 0 */
    double a, b;      /* the interval I = [a, b], a < b, both finite */
    double p[8];      /* parameters, see pwl_kind */
} pwl_func;

/* Which CPWL approximation of f the vertex values define (Section II-B). */
typedef enum {
    PWL_INTERP = 0,  /* linear interpolant pi_T f: v_i = f(x_i)            (Eq. 3)    */
    PWL_PROJECT = 1  /* L2 orthogonal projection P_T f: M c = b, v_i = c_i  (Eqs. 4-6) */
} pwl_form;

/* Storage type of a vertex-value table or of a query / result stream.  The
 * interpolation arithmetic is FP32 in every case. */
typedef enum { PWL_FP32 = 0, PWL_BF16 = 1, PWL_FP16 = 2 } pwl_dtype;

/* Precision of the integrands of the design and projection steps (the
 * density |f''|^{2/5} and f at quadrature nodes).  Prefix sums, knot
 * inversion, quadrature sums and the tridiagonal solve are FP64 in both. */
typedef enum { PWL_PREC_FP64 = 0, PWL_PREC_FP32 = 1 } pwl_precision;

typedef struct pwl_table_s* pwl_table;
typedef struct pwl_batch_s* pwl_batch;
typedef struct pwl_channels_s* pwl_channels;

/* ------------------------------------------------------------------------ */
/* Library                                                                   */
/* ------------------------------------------------------------------------ */

/* Thread-local description of the last failure of a call on this thread. */
const char* pwl_last_error(void);

/* ABI version (major * 10000 + minor * 100 + patch). */
int32_t pwl_version(void);

/* Fills *out with the descriptor of a sampled function (PWL_F_SAMPLED):
 * n_samples >= 4 FP64 samples of f at a + j (b - a)/(n_samples - 1) in
 * device memory (d_samples, 8-byte aligned, owned by the caller).  Host
 * only; errors: PWL_EINVAL (NULL, n_samples < 4, a >= b, non-finite a, b).  */
pwl_status pwl_func_sampled(double a, double b, const double* d_samples, int64_t n_samples, pwl_func* out);

/* ------------------------------------------------------------------------ */
/* Design: knots of the nearly optimal partition T* (Section III-B)          */
/* ------------------------------------------------------------------------ */

/* Bytes of workspace pwl_design needs for n_intervals and m_cells. */
size_t pwl_design_workspace_size(int64_t n_intervals, int64_t m_cells);

/* Knots x_0..x_N of T* for f (Eqs. 16-18): the local knot density
 * |f''|^{2/5} is sampled at the midpoints t_k = a + (k + 1/2)(b - a)/M of M
 * uniform cells (precision per `precision`), prefix-summed in FP64 into
 * G_k = delta * sum_{j<k} d_j (the numerator of Eq. 18 by the midpoint rule),
 * and inverted: x_0 = a, x_N = b, and for 0 < i < N, with tau_i = i G_M / N,
 * the cell is the largest k with G_k <= tau_i and d_k > 0 and
 * x_i = a + k delta + (tau_i - G_k) / d_k.  If G_M == 0 (f linear on I) the
 * uniform partition is returned.
 *   f          host pointer to the function descriptor
 *   n_intervals N >= 1
 *   m_cells    M >= 1 density cells; 0 selects 64 N
 *   precision  pwl_precision of the density samples
 *   d_knots    device, N+1 doubles (output, strictly increasing)
 * Errors: PWL_EINVAL for a bad descriptor, sizes or workspace.             */
pwl_status pwl_design(const pwl_func* f, int64_t n_intervals, int64_t m_cells, int32_t precision,
                      double* d_knots, void* d_workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Vertex values (Section II-B)                                              */
/* ------------------------------------------------------------------------ */

size_t pwl_project_workspace_size(int64_t n_intervals);

/* Vertex values of pi_T f (form PWL_INTERP, v_i = f(x_i), Eq. 3) or of
 * P_T f (form PWL_PROJECT, Eqs. 4-6): b_i = <f, phi_i> by quad_points-point
 * Gauss-Legendre quadrature on every interval (1 <= quad_points <= 16; 0
 * selects 8), the tridiagonal Gram matrix M_ii = (h_i + h_{i+1})/3,
 * M_{i,i+1} = h_{i+1}/6, and M c = b solved in FP64 by cyclic reduction.
 *   d_knots   device, N+1 strictly increasing doubles (e.g. from pwl_design)
 *   d_values  device, N+1 doubles (output)
 * The workspace (pwl_project_workspace_size bytes) also carries the function
 * descriptor to the device, so it is needed for both forms.                */
pwl_status pwl_project(const pwl_func* f, const double* d_knots, int64_t n_intervals,
                       int32_t form, int32_t quad_points, int32_t precision, double* d_values,
                       void* d_workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* A priori errors and the N for a target error (Results 4-6, Section III-B) */
/* ------------------------------------------------------------------------ */

/* The two integrals the error results need, by the midpoint rule on m_cells
 * uniform cells t_k = a + (k + 1/2)(b - a)/M (the discretisation of
 * pwl_design) in FP64:
 *   d_out[0] = integral over [a, b] of |f''|^{2/5}   (Result 4)
 *   d_out[1] = integral over [a, b] of f''^2         (Result 6, ||f''||^2)
 *   f        host pointer to the function descriptor
 *   m_cells  M >= 1; 0 selects 2^20
 *   d_out    device, 2 doubles (overwritten)
 * Asynchronous on stream.  Errors: PWL_EINVAL (descriptor, sizes, NULL).    */
pwl_status pwl_error_constants(const pwl_func* f, int64_t m_cells, double* d_out, void* stream);

/* Predicted L2 error of the CPWL approximation with N intervals (host only):
 *   form PWL_INTERP, uniform = 0 (T*, Result 4):
 *       (int |f''|^{2/5})^{5/2} / (N^2 sqrt(120))
 *   form PWL_INTERP, uniform = 1 (Result 6):
 *       (b - a)^2 ||f''|| / (N^2 sqrt(120)),  ||f''|| = sqrt(int f''^2)
 *   form PWL_PROJECT: the same divided by sqrt(6) (Result 5; the per-interval
 *       ratio of Results 2-3 holds on any partition).
 *   int_f2_25, int_f2_sq  the two integrals of pwl_error_constants (>= 0)
 *   a, b                  the interval (a < b, finite)
 *   err_out               host, one double
 * Asymptotic in N (large N); errors: PWL_EINVAL.                            */
pwl_status pwl_predicted_error(double int_f2_25, double int_f2_sq, double a, double b, int64_t n_intervals,
                               int32_t form, int32_t uniform, double* err_out);

/* Smallest N whose predicted error (as pwl_predicted_error) is <= target_l2
 * (host only).  n_out: host, one int64.  Errors: PWL_EINVAL (arguments, or a
 * target needing more intervals than pwl_design accepts).                  */
pwl_status pwl_n_for_error(double int_f2_25, double int_f2_sq, double a, double b, double target_l2, int32_t form,
                           int32_t uniform, int64_t* n_out);

/* ------------------------------------------------------------------------ */
/* Device representation of a CPWL function (inputs of Algorithm 1)          */
/* ------------------------------------------------------------------------ */

/* Builds a table from FP64 knots and values (device arrays of N+1).  Knots
 * are rounded to FP32 and values to `value_dtype` (round to nearest); the
 * table evaluates exactly that CPWL function.  For evaluation it adds a
 * uniform cell index over [x_0, x_N]: k_cells cells (0 = automatic), each
 * holding the knot at or before it with the slopes on both sides, so that
 * Algorithm 1's search step is one lookup.
 * Synchronizes `stream` (it validates the rounded knots and sizes the
 * index).  Errors: PWL_EINVAL if the rounded knots are not strictly
 * increasing or a value or slope is not finite.                            */
pwl_status pwl_table_build(const double* d_knots, const double* d_values, int64_t n_intervals,
                           int32_t value_dtype, int64_t k_cells, pwl_table* out, void* stream);

/* Rebuilds the table in place from new FP64 knots and values (same N, value
 * dtype and cell count), asynchronously on `stream` and without allocating:
 * the call a training or design loop makes every step.  The knots must stay
 * strictly increasing after rounding to FP32, every value and slope finite,
 * and the end knots x_0, x_N must round to the FP32 values of the build (the
 * cell grids span the built [x_0, x_N]; interior knots may move freely).
 * This call does not check; pwl_table_check reports a violation, after
 * which evaluation is unspecified until a valid update.  The comparison
 * path's texture (pwl_eval_variant mode 1), if created, is refreshed on
 * `stream` too.  It must not overlap other work on the same table.          */
pwl_status pwl_table_update(pwl_table t, const double* d_knots, const double* d_values, void* stream);

/* Status of the last build or update: PWL_EINVAL if the rounded knots were
 * not strictly increasing, a value or slope not finite, or an update moved
 * an end knot.  Synchronizes `stream`.                                      */
pwl_status pwl_table_check(pwl_table t, void* stream);

pwl_status pwl_table_destroy(pwl_table t);

typedef struct {
    int64_t n_intervals;   /* N */
    int64_t k_cells;       /* cells of the uniform index */
    int64_t n_chain;       /* extra records for cells holding more than one knot */
    int32_t value_dtype;   /* pwl_dtype of the stored values */
    int32_t reserved;
    float a, b;            /* x_0, x_N as stored (FP32) */
    const float* d_knots;  /* device, N+1 FP32 knots used by every kernel */
    const void* d_values;  /* device, N+1 values in value_dtype */
    size_t eval_smem_bytes;     /* shared memory one forward CTA stages */
    size_t backward_smem_bytes; /* shared memory one backward CTA stages */
    int32_t layout;             /* forward index pwl_eval uses: 0 = 8-byte cell records with two
                                   side records per knot, 1 = 16-byte records, 2 = 8-byte cell
                                   records with one side record per knot */
    int32_t reserved2;
} pwl_table_info;

pwl_status pwl_table_get_info(pwl_table t, pwl_table_info* info);

/* ------------------------------------------------------------------------ */
/* Evaluation (Algorithm 1)                                                  */
/* ------------------------------------------------------------------------ */

/* y[q] = v(x[q]) for q < m (Algorithm 1), the interpolation in FP32.  x and
 * y are device arrays of m elements of io_dtype (PWL_FP32, PWL_BF16 or
 * PWL_FP16; the same for both).  x outside [x_0, x_N] is clamped (y = v_0 or
 * v_N); x = x_N uses the last interval; NaN gives NaN.  Any alignment; the
 * 16-byte vector path is used when x and y share their alignment.  x and y
 * may be the same array.                                                   */
pwl_status pwl_eval(pwl_table t, const void* d_x, void* d_y, int64_t m, int32_t io_dtype,
                    void* stream);

/* Comparison paths for the measurements of Section V-A (Table I):
 *   mode 0: Algorithm 1 with the search of Section IV: a binary search over
 *           the FP32 knots in shared memory, unrolled at compile time for
 *           2^L >= N+1 knot slots (L <= 14, so N <= 16383) with selects in
 *           place of branches; delta by a division; (1 - delta) v_{i-1} +
 *           delta v_i (O(log N) per query);
 *   mode 1: the same interval lookup as pwl_eval, then the texture unit's
 *           linear filter at coordinate i - 1 + delta + 1/2 over the values
 *           (Section IV-B); the filter weight is fixed point (8 fractional
 *           bits), so results differ from pwl_eval by up to |v_i - v_{i-1}|/256;
 *   mode 2, 3: pwl_eval forced to its 8-byte or 16-byte cell index (it
 *           otherwise picks one per table, see pwl_table_info.layout);
 *   mode 6: pwl_eval forced to the 8-byte cell index with one side record
 *           per knot (layout 2; the same results as mode 2 on the same cells);
 *   mode 4: the search of mode 0, then the texture filter of mode 1 (Table
 *           I's optimized partition with hardware interpolation);
 *   mode 5: the uniform-partition lookup of Section IV with the texture
 *           filter: coordinate (x - x_0) N / (x_N - x_0) + 1/2, no search;
 *           correct only for a table whose knots are uniform (e.g. built
 *           from x_i = a + i (b - a)/N), up to the 8-bit weight.
 * x, y: device FP32 arrays of m elements.  The texture of modes 1, 4, 5 is
 * created on first use (an allocation) and refreshed by pwl_table_update.  */
pwl_status pwl_eval_variant(pwl_table t, int32_t mode, const float* d_x, float* d_y, int64_t m,
                            void* stream);

/* Compute ceiling of Algorithm 1 (the analogue of the paper's synthetic
 * timings, Table I): the table is evaluated at m queries generated in
 * registers, with no query read from memory and no result written.  Query q
 * (0 <= q < m <= 2^32) is x_q = u_q (b - a) + a in FP32 (a product and a
 * sum, each rounded to nearest), where a, b are the table's FP32 end knots
 * and u_q = (lowbias32((q + seed) mod 2^32) >> 8) / 2^24, lowbias32 being
 * the 32-bit integer hash of the hash-prospector project (x ^= x >> 16;
 * x *= 0x7feb352d; x ^= x >> 15; x *= 0x846ca68b; x ^= x >> 16).  Every CTA
 * adds the FP32 sum of its results (in an unspecified order) to *d_sum, a
 * device FP64 word the caller zeroes: a checksum that keeps the work live.  */
pwl_status pwl_eval_synthetic(pwl_table t, uint32_t seed, int64_t m, double* d_sum, void* stream);

/* pwl_eval_synthetic for the comparison paths of pwl_eval_variant (modes
 * 0..6, same queries and checksum): the compute ceilings of Table I's rows
 * on this GPU (binary search vs cell index, lerp vs texture filter).       */
pwl_status pwl_eval_synthetic_variant(pwl_table t, int32_t mode, uint32_t seed, int64_t m, double* d_sum,
                                      void* stream);

/* ------------------------------------------------------------------------ */
/* Direct evaluation of f: the comparison systems of Section V               */
/* ------------------------------------------------------------------------ */

/* y[q] = f(x[q]) computed directly in FP32, the alternatives the paper
 * times against the CPWL evaluation (Table I; Sections V-B and V-C):
 *   PWL_F_GAUSSIAN    method 0: A expf(-u^2/2), u = (x - mu)(1/s)
 *                     method 1: the same with the SFU's __expf
 *   PWL_F_LORENTZIAN  method 0: A / (1 + u^2), u = (x - x0)(1/g), IEEE division
 *                     method 1: the same with __fdividef (fast division)
 *   PWL_F_BESSEL_J0   method 0: A j0f(alpha x) (the CUDA math library)
 *                     method 1: the first term of the asymptotic expansion,
 *                     A sqrt(2/pi) rsqrtf(z) __cosf(z - pi/4), z = alpha x
 *                     (valid for z >> 1/4; its error decays like z^{-3/2};
 *                     z <= 0 gives inf or NaN)
 * with the parameters of pwl_kind (A, mu, 1/s, x0, 1/g, alpha and
 * A sqrt(2/pi) formed in FP64 and rounded to FP32 once).  No clamping to
 * [a, b]: f is evaluated at x as given.  x, y: device FP32 arrays of m
 * elements (any alignment; y may be x), streamed like pwl_eval.  Errors:
 * PWL_EINVAL (descriptor, method, sizes, NULL), PWL_ENOTSUP (other kinds).   */
pwl_status pwl_direct_eval(const pwl_func* f, int32_t method, const float* d_x, float* d_y, int64_t m,
                           void* stream);

/* The compute ceiling of pwl_direct_eval: f at the m register-generated
 * queries of pwl_eval_synthetic (x_q = u_q (b - a) + a with a, b the FP32
 * roundings of f->a, f->b), every CTA adding the FP32 sum of its results to
 * *d_sum (device FP64 word, zeroed by the caller).                          */
pwl_status pwl_direct_synthetic(const pwl_func* f, int32_t method, uint32_t seed, int64_t m, double* d_sum,
                                void* stream);

/* Backward of pwl_eval for upstream gradients gy (FP32, m elements):
 *   gx[q] = gy[q] * s_i (s_i the slope of x[q]'s interval; 0 if clamped)
 *   g_values[j] += sum over queries of gy * dy/dv_j  (N+1 FP32, or NULL)
 *   g_knots[j]  += sum over queries of gy * dy/dx_j  (N+1 FP32, or NULL)
 * with dy/dv_{i-1} = 1 - delta, dy/dv_i = delta, dy/dx_{i-1} = -s (1 - delta),
 * dy/dx_i = -s delta; a clamped query adds gy to g_values[0] or [N] only.
 * g_values / g_knots are accumulated into (the caller zeroes them).  Each
 * CTA accumulates the per-interval sums in 32-bit fixed point with integer
 * shared-memory atomics: its unit is 2^-F with 2^F ~ 2^23 / (geometric mean
 * of the |gy| among its first queries; F limited to [-60, 126], so that
 * gradients of typical magnitude below ~1e-31 get a coarser unit), each
 * term is rounded to the unit once (absolute error <= 2^-(F+1)), integer
 * wraps and multiples of 2^32
 * units are counted exactly (in FP32 multiples of 2^(32-F), exact below
 * 2^24 of them per CTA and interval), and terms of 2^62 units or more (or
 * inf, NaN) are summed in FP32.  The
 * CTA partial sums are then reduced in a fixed order in FP64; run-to-run
 * differences come only from the order of the FP32-summed terms (none for
 * gradients of moderate range).  gx may alias gy.
 * Workspace: pwl_eval_backward_workspace_size(t) bytes.                    */
size_t pwl_eval_backward_workspace_size(pwl_table t);
pwl_status pwl_eval_backward(pwl_table t, const float* d_x, const float* d_gy, float* d_gx,
                             float* d_g_values, float* d_g_knots, int64_t m, void* d_workspace,
                             size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Batches: many independent functions, each with its own partition          */
/* ------------------------------------------------------------------------ */

/* A batch holds F functions f_0..f_{F-1}, function f with its own interval
 * I_f and N_f intervals (Section II-B for each).  Its device arrays are
 * concatenated in function order: knots and values of function f occupy
 * entries koff[f] .. koff[f] + N_f, koff[f] = sum_{g<f} (N_g + 1).  Each
 * phase is one fixed sequence of launches over all functions, enqueued
 * without host synchronisation, so that design, projection, index build and
 * evaluation can be captured in one CUDA graph and replayed.
 *   funcs          host, F descriptors (validated as for pwl_design)
 *   n_intervals    host, F values N_f in [1, 65535]
 *   m_per_interval density cells per interval of the design step
 *                  (M_f = m_per_interval N_f); 0 selects 64
 *   cells_per_knot cells of each function's evaluation index per knot
 *                  (0 selects 3), reduced where the index would not fit one
 *                  CTA's shared memory
 * Allocates all device memory of the batch (synchronously); the batch owns
 * it until pwl_batch_destroy.  Errors: PWL_EINVAL (sizes, a descriptor),
 * PWL_ENOMEM / PWL_ECUDA (allocation).                                      */
pwl_status pwl_batch_create(const pwl_func* funcs, const int64_t* n_intervals, int64_t n_funcs,
                            int64_t m_per_interval, int64_t cells_per_knot, pwl_batch* out);
pwl_status pwl_batch_destroy(pwl_batch b);

/* Knots of T* for every function (pwl_design per function, Eqs. 16-18, with
 * M_f cells): the knots land in the batch's FP64 knot array.               */
pwl_status pwl_batch_design(pwl_batch b, int32_t precision, void* stream);

/* Vertex values of every function (pwl_project per function, Eqs. 3-6) from
 * the batch's knots into its FP64 value array.                             */
pwl_status pwl_batch_project(pwl_batch b, int32_t form, int32_t quad_points, int32_t precision,
                             void* stream);

/* Evaluation index of every function from the batch's FP64 knots and values
 * (rounded to FP32; the CPWL function evaluated is exactly that rounded
 * one).  Call after pwl_batch_design / pwl_batch_project, or after writing
 * the FP64 arrays through pwl_batch_get_info.  Does not check the rounded
 * knots (pwl_batch_check does).                                            */
pwl_status pwl_batch_build(pwl_batch b, void* stream);

/* PWL_EINVAL if the last build found a function whose rounded knots are not
 * strictly increasing or a knot or value not finite (message names the
 * first one); evaluation of such a function is unspecified.  PWL_ETIMEOUT
 * if an evaluation since the last check gave up waiting for a staging copy
 * (its results are then incomplete); the check clears that flag.
 * Synchronizes `stream`.                                                    */
pwl_status pwl_batch_check(pwl_batch b, void* stream);

/* Plans evaluation for a query layout: function f's queries are
 * x[query_offsets[f]] .. x[query_offsets[f+1] - 1] (host array of F+1
 * non-decreasing offsets, query_offsets[0] = 0).  The concatenated stream
 * is cut into one contiguous range per CTA of a persistent grid, of about
 * equal cost; a CTA stages a function's index in shared memory when its
 * share of the function's queries times stage_min is at least the index
 * bytes (stage_min 0: never stage; -1: keep the current value, initially
 * 16).  shape (-1 keeps the current one, initially 0):
 *   0  one 1024-thread CTA per SM staging the records with its threads (an
 *      index of up to all of the CTA's shared memory);
 *   1  as 0, the queries streamed through a 4-slot cp.async ring in shared
 *      memory (the index gets the rest);
 *   2  two 512-thread CTAs per SM, each staging with its threads (an index
 *      of up to half of the SM's shared memory);
 *   3  no staging: every piece reads its records through L1 (stage_min is
 *      ignored);
 *   4  one 1024-thread CTA per SM with two record buffers: a bulk copy
 *      (cp.async.bulk) brings the next piece's records while the CTA
 *      streams the current piece (an index of up to half of the CTA's
 *      shared memory).
 * A function whose index exceeds the shape's budget is read through L1.
 * Allocates the plan (synchronously; the previous plan is freed).  A wait
 * for a bulk copy gives up after 1 s; pwl_batch_check then reports
 * PWL_ETIMEOUT.                                                             */
pwl_status pwl_batch_plan(pwl_batch b, const int64_t* query_offsets, int32_t shape, int64_t stage_min);

/* y[q] = v_f(x[q]) for every planned query (Algorithm 1 per function, the
 * same arithmetic, clamping and NaN rule as pwl_eval): one persistent
 * launch.  x, y: device FP32 arrays of query_offsets[F] elements, 16-byte
 * aligned; y may be x.                                                      */
pwl_status pwl_batch_eval(pwl_batch b, const float* d_x, float* d_y, void* stream);

/* Autotuner: times pwl_batch_eval on the caller's x and y (reps timed
 * launches per candidate after one warm-up) for every CTA shape (0..4) and
 * staging threshold stage_min in {0, 4, 16, 64}, and keeps the fastest plan.
 * timings_ms: host array of 20 floats receiving the mean launch time of
 * candidate (shape, threshold) at index 4 shape + threshold position, or
 * NULL.  Writes y; synchronizes `stream`; must not run during stream
 * capture.                                                                  */
pwl_status pwl_batch_autotune(pwl_batch b, const float* d_x, float* d_y, int32_t reps, float* timings_ms,
                              void* stream);

typedef struct {
    int64_t n_funcs;
    int64_t total_knots;     /* sum of N_f + 1 */
    int64_t total_cells;     /* cells of all evaluation indexes */
    int64_t index_bytes;     /* bytes of all evaluation indexes */
    int64_t total_queries;   /* of the current plan (0 before pwl_batch_plan) */
    int32_t eval_grid;       /* CTAs of the evaluation launch */
    int32_t eval_threads;    /* threads per CTA */
    int32_t eval_shape;
    int32_t reserved;
    int64_t n_items;         /* (function, query range) pieces of the plan */
    int64_t n_staged;        /* pieces that stage their function's index */
    int64_t stage_min;
    int64_t smem_bytes;      /* dynamic shared memory of the evaluation launch */
    const int64_t* d_knot_offsets; /* device, F+1 offsets koff */
    double* d_knots;         /* device, FP64 knots (written by pwl_batch_design) */
    double* d_values;        /* device, FP64 values (written by pwl_batch_project) */
    const float* d_knots_fp32;  /* device, FP32 knots of the last build */
    const float* d_values_fp32; /* device, FP32 values of the last build */
} pwl_batch_info;

pwl_status pwl_batch_get_info(pwl_batch b, pwl_batch_info* info);

/* ------------------------------------------------------------------------ */
/* Channel-wise maps: one CPWL function per channel (Algorithm 1 per element) */
/* ------------------------------------------------------------------------ */

/* y[r, c] = v_c(x[r, c]) for a row-major x[rows, n_channels], where channel
 * c is the CPWL function with FP32 knots d_knots[c, 0..N] and values
 * d_values[c, 0..N] (device arrays [n_channels, N+1], e.g. learnable
 * parameters).  Each CTA builds the cell index of 8 channels in shared
 * memory (k_cells cells per channel of 16 bytes each, 0 selects 4 (N+1) as
 * far as the CTA's shared memory allows; cells holding several knots are
 * walked).  io_dtype PWL_FP32 or PWL_BF16 (x and y alike); the arithmetic
 * is FP32; clamping and NaN as in pwl_eval.  Knots must be strictly
 * increasing per channel: a violation sets bit 0 of the device word
 * *d_status (the caller zeroes it; results are then unspecified).
 * Errors: PWL_ENOTSUP if 8 channels' index does not fit a CTA
 * (128 (k_cells + N + 1) bytes).                                           */
pwl_status pwl_channels_forward(const float* d_knots, const float* d_values, int64_t n_channels,
                                int64_t n_intervals, int64_t k_cells, const void* d_x, void* d_y,
                                int64_t rows, int32_t io_dtype, int32_t* d_status, void* stream);

/* Backward of pwl_channels_forward (FP32 only): gx[r, c] = gy[r, c] * s,
 * and for every channel d_g_values[c, j] += sum over rows of gy dy/dv_j,
 * d_g_knots[c, j] += sum of gy dy/dx_j (the formulas of pwl_eval_backward;
 * either may be NULL; accumulated with FP32 atomics, order-dependent at FP32
 * rounding).  k_cells: 0 selects 2 (N+1).                                  */
pwl_status pwl_channels_backward(const float* d_knots, const float* d_values, int64_t n_channels,
                                 int64_t n_intervals, int64_t k_cells, const float* d_x, const float* d_gy,
                                 float* d_gx, float* d_g_values, float* d_g_knots, int64_t rows,
                                 int32_t* d_status, void* stream);

/* ------------------------------------------------------------------------ */
/* Failure injection: tests of the error paths (no counterpart in the paper;  */
/* nothing here faults or hangs a GPU)                                        */
/* ------------------------------------------------------------------------ */

/* Makes the library's device allocations fail: succeed_first = n >= 0 lets
 * the next n allocations (cudaMalloc / cudaMallocArray inside pwl_table_build,
 * pwl_batch_create, pwl_batch_plan and the texture of pwl_eval_variant)
 * through and fails every later one with PWL_ENOMEM, until the hook is reset
 * with succeed_first < 0.  A failing call releases what it had allocated and
 * leaves its output handle NULL (or the existing plan / texture unchanged).
 * Process-wide; host only; always PWL_OK.                                   */
pwl_status pwl_test_fail_allocations(int64_t succeed_first);

/* Makes the bounded waits of the asynchronous batch evaluation (shape 4 of
 * pwl_batch_plan) run out, to test their timeout path.  withhold = 1: every
 * staging barrier of the following pwl_batch_eval launches expects one
 * arrival more than the kernel makes, so the first wait for a staging copy
 * of each CTA gives up after wait_limit_ns; the CTA then makes the withheld
 * arrival, waits (bounded) for its bulk copies to land, stops, and
 * pwl_batch_check reports PWL_ETIMEOUT (its results are incomplete).
 * withhold = 0 restores normal operation; wait_limit_ns 0 restores the
 * default limit of 1 s (at most 1 s).  Host only; takes effect at the next
 * pwl_batch_eval.  Errors: PWL_EINVAL (NULL batch, arguments).             */
pwl_status pwl_batch_inject_wait_timeout(pwl_batch b, int32_t withhold, uint64_t wait_limit_ns);

/* pwl_eval_backward for callers that cannot allocate device memory (the
 * paper has no counterpart; this is a library concern): real-time loops that
 * fix their memory at start-up, code called back from a host framework that
 * owns all device memory, and callers with no workspace to lend.  It takes
 * the same inputs and outputs as pwl_eval_backward but no workspace: its
 * per-CTA partial sums go to a static device array of 2^21 floats (8 MiB)
 * that every GPU which loads the library holds until the process exits.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - N must satisfy 2 (N + 2) * (SM count) <= 2^21 (N <= 6896 on a 152-SM
 *     GB300); larger tables are rejected with PWL_EINVAL and a message.
 *   - Every call shares the one array and overwrites what it uses, so calls
 *     whose work overlaps on the GPU (other streams, other threads) race:
 *     serialise them.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.        */
pwl_status pwl_eval_backward_noalloc(pwl_table t, const float* d_x, const float* d_gy, float* d_gx,
                                     float* d_g_values, float* d_g_knots, int64_t m, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PWL_H */
