// pwl_table.cuh -- internal helpers around pwl_table: cell-count choice,
// shared-memory budgets of the streaming kernels and their launch shapes.
#pragma once

#include <algorithm>

#include "pwl_common.cuh"

namespace pwl {

// Forward index: K 8-byte cell records plus 2 (N+1) 8-byte side records.
inline size_t forward_side_bytes(int64_t N) { return sizeof(float2) * 2 * (size_t)(N + 1); }
// The side records are staged in shared memory when they leave room for at
// least 1024 cell records; otherwise the kernel reads them from global memory.
inline bool forward_side_staged(int64_t N)
{
    return forward_side_bytes(N) + 8 * 1024 <= device_info().smem_optin;
}
inline size_t eval8_smem_bytes(const pwl_table_s* t)
{
    return sizeof(float2) * (size_t)t->K + (forward_side_staged(t->N) ? forward_side_bytes(t->N) : 0);
}
// 8-byte index with one side record per knot ({v_k, s_{k+1}}; a query left
// of knot k takes s_k from the record of knot k - 1): K cell records plus
// N+1 side records, always staged.
inline size_t eval8c_smem_bytes(const pwl_table_s* t)
{
    return sizeof(float2) * ((size_t)t->K + (size_t)(t->N + 1));
}
// 16-byte index for the forward path: K_b cells and reserved chain records
inline int64_t eval16_smem_records(const pwl_table_s* t)
{
    const int64_t cap = (int64_t)(device_info().smem_optin / sizeof(float4));
    return std::min<int64_t>(t->Kb + t->chain_reserve_b, cap);
}
inline size_t eval16_smem_bytes(const pwl_table_s* t) { return sizeof(float4) * (size_t)eval16_smem_records(t); }

// cells of an 8-byte index that fit `budget` bytes next to the side records
int64_t forward_cell_capacity(int64_t N, size_t budget);
int64_t backward_cell_capacity(int64_t N);
void choose_cells(pwl_table t, float hmin, int64_t requested);
// Re-copies the rounded values into the texture of the comparison path, if
// the table has one (after an in-place update), on stream s.
pwl_status refresh_texture(pwl_table t, cudaStream_t s);

// Backward: K_b + reserved chain records, N+2 reciprocal lengths and
// 2 (N+2) int32 accumulators per copy.  The accumulators have L copies (lane l
// of every warp adds into copy l mod L, accumulator (i, copy) at i L + copy,
// so that one warp's atomics spread over L bank classes and never share an
// address within a copy group): L = 32, 16, 8, 4, 2 or 1, the largest that
// fits next to all the records.  Chain records beyond the reserve are read
// from global memory.
// (plus 16 bytes after the accumulators for the kernel's two scalars)
constexpr size_t kBwdScalarSmem = 16;
inline int backward_lanes(const pwl_table_s* t)
{
    const size_t optin = device_info().smem_optin;
    const size_t rec = 16 * (size_t)(t->Kb + t->chain_reserve_b), n2 = (size_t)(t->N + 2);
    for (int L = 32; L > 1; L /= 2)
        if (rec + 4 * n2 + 8 * n2 * (size_t)L + kBwdScalarSmem <= optin) return L;
    return 1;
}
inline size_t backward_fixed_smem(const pwl_table_s* t)
{
    return (4 + 8 * (size_t)backward_lanes(t)) * (size_t)(t->N + 2) + kBwdScalarSmem;
}
// Record copies R (1, 2, 4 or 8; the largest that fits next to the
// accumulators with every record staged).  A warp's 16-byte gathers are served
// a quarter warp (8 lanes) at a time, and 8 random records of one copy
// collide in ~2.5 of the 8 16-byte bank groups; copy g of record c sits at
// index c R + g and lane l reads copy l mod R, so with R = 8 the lanes of a
// quarter warp always hit 8 different bank groups.
inline int backward_record_copies(const pwl_table_s* t)
{
    const size_t optin = device_info().smem_optin;
    const size_t fixed = backward_fixed_smem(t);
    const size_t rec = 16 * (size_t)(t->Kb + t->chain_reserve_b);
    for (int R = 8; R > 1; R /= 2)
        if (fixed + rec * (size_t)R <= optin) return R;
    return 1;
}
inline int64_t backward_smem_records(const pwl_table_s* t)
{
    const size_t optin = device_info().smem_optin;
    const size_t fixed = backward_fixed_smem(t);
    if (fixed + 16 * 64 > optin) return -1;  // does not fit: unsupported
    const int64_t cap = (int64_t)((optin - fixed) / (sizeof(float4) * (size_t)backward_record_copies(t)));
    return std::min<int64_t>(t->Kb + t->chain_reserve_b, cap);
}
inline size_t backward_smem_bytes(const pwl_table_s* t)
{
    const int64_t r = backward_smem_records(t);
    return r < 0 ? 0 : sizeof(float4) * (size_t)r * (size_t)backward_record_copies(t) + backward_fixed_smem(t);
}

// Persistent grid of a kernel: resident CTAs per SM (registers, shared
// memory, threads) times the SM count, with the kernel's dynamic shared
// memory limit raised to smem first (cached host calls).
template <typename Kern>
inline cudaError_t occupancy_grid(Kern kern, int threads, size_t smem, int* grid)
{
    return occupancy_grid_fn(reinterpret_cast<const void*>(kern), threads, smem, grid);
}

}  // namespace pwl
