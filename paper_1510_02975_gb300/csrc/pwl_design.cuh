// pwl_design.cuh -- internal interface of the batched design and projection
// kernels (one function is a batch of one).
#pragma once

#include "pwl_common.cuh"

namespace pwl {

constexpr int kMaxIntervals = 1048575;

// 1/d for a positive normal FP64 d by Newton's method for the reciprocal,
// r <- r + r (1 - d r), from the hardware's approximate reciprocal
// (rcp.approx.ftz.f64); each step doubles the correct bits, two reach FP64
// rounding.  Five FP64 operations against about twice that for a division
// (the Gram solves and the table build's slopes and reciprocal lengths).
__device__ __forceinline__ double recip_newton(double d)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
    double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
    e = fma(-d, r, 1.0);
    return fma(r, e, r);
}

// F functions; function f owns knots koff[f] .. koff[f+1]-1 (N_f + 1 of them),
// density cells moff[f] .. moff[f+1]-1 (M_f), chunks choff[f] .. choff[f+1]-1,
// and G entries moff[f] + f .. moff[f+1] + f (M_f + 1).
// Which kinds a plan holds: the hot kernels are compiled once for the
// analytic kinds and once for sampled functions (whose FP64 interpolation
// would otherwise weigh on the analytic loops' registers); a launch runs the
// instantiations its plan needs.  0 means both.
constexpr int kKindsAnalytic = 1;
constexpr int kKindsSampled = 2;
inline int plan_kinds(int kinds) { return kinds ? kinds : (kKindsAnalytic | kKindsSampled); }
inline int kinds_of(const pwl_func* f, int64_t n)
{
    int k = 0;
    for (int64_t i = 0; i < n; ++i) k |= f[i].kind == PWL_F_SAMPLED ? kKindsSampled : kKindsAnalytic;
    return k;
}

struct DesignPlan {
    int F;
    int precision;
    int kinds;  // kKindsAnalytic | kKindsSampled of the functions (0: both)
    const pwl_func* funcs;
    const int64_t* koff;
    const int64_t* moff;
    const int64_t* choff;
    int64_t total_knots, total_cells, total_chunks;
    double* d;      // total_cells densities
    double* G;      // total_cells + F cumulative values
    double* csum;   // total_chunks partial sums
    double* cbase;  // total_chunks exclusive chunk bases
    double* stot;   // F totals (sum of d over the function)
    double* knots;  // total_knots output
    // fused per-function path (batches)
    const int* order;  // F function indices, largest M first
    int* clast;        // total_chunks: last cell of positive density in the chunk (local index), or -1;
                       // must not overlap d (the FP32 fused kernel keeps FP32 densities there)
};

int64_t design_chunks(int64_t M);
size_t design_scratch_bytes(int64_t F, int64_t total_cells, int64_t total_chunks);
void design_carve_scratch(DesignPlan& p, void* scratch);
pwl_status design_launch(const DesignPlan& p, cudaStream_t s);
// One persistent launch for a batch: each CTA designs whole functions (in
// p.order); needs p.order and p.clast, writes p.csum, p.cbase and p.knots.
pwl_status design_fused_launch(const DesignPlan& p, cudaStream_t s);

// Projection: F functions with knots at koff (device), values out.
struct ProjectPlan {
    int F;
    int precision;
    int kinds;  // kKindsAnalytic | kKindsSampled of the functions (0: both)
    int form;
    int max_rows;          // max over f of N_f + 1
    int64_t total_knots;
    int64_t total_intervals;
    const pwl_func* funcs;
    const int64_t* koff;
    const double* knots;
    double* values;
    double2* lr;           // per interval: (int f phi_left, int f phi_right)
    double* cr;            // 4 * total_knots doubles of solver scratch (used when rows do not fit smem)
    int solver;            // 0: cyclic reduction, one CTA per function; 1: partitioned Thomas, one warp per function
    const int* order;      // solver 1: the order in which warps take the functions (NULL: 0..F-1)
};

struct GaussLegendre {
    int Q;
    double x[16];   // nodes on [-1, 1]
    double w[16];   // weights
    double wl[16];  // w (1 - x) / 2: the weight times the left hat phi_{j-1} at the node
    double wr[16];  // w (1 + x) / 2: the weight times the right hat phi_j at the node
    float xf[16];   // nodes rounded to FP32
    float wlh[16], wll[16], wrh[16], wrl[16];  // wl, wr split into FP32 pairs hi + lo
};
const GaussLegendre& gauss_legendre_rule(int Q);

size_t project_scratch_bytes(int64_t total_knots, int64_t total_intervals);
void project_carve_scratch(ProjectPlan& p, void* scratch);
pwl_status project_launch(const ProjectPlan& p, const GaussLegendre& gl, cudaStream_t s);

}  // namespace pwl
