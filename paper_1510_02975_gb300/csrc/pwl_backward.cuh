// pwl_backward.cuh -- internal interface of the backward kernels.
#pragma once

#include "pwl_table.cuh"

namespace pwl {

struct BwdShape {
    int64_t n_smem;    // records staged per CTA (-1: table too large)
    size_t smem;       // dynamic shared memory per CTA
    int threads;
    int grid;          // persistent grid (maximum CTAs of one launch)
    size_t workspace;  // bytes of per-CTA partial sums for `grid` CTAs
    cudaError_t err;   // the CUDA error that made n_smem -1, if any
};

BwdShape backward_shape(pwl_table t);

// Streams (x, gy) -> gx with `grid` CTAs, writes per-CTA partial sums into
// `partials` (grid rows of 2 (N + 2) floats) and, if g_values or g_knots is
// non-NULL, reduces them into those arrays.
pwl_status backward_launch(pwl_table t, const float* x, const float* gy, float* gx, float* g_values,
                           float* g_knots, int64_t m, float* partials, int grid, cudaStream_t s);

}  // namespace pwl
