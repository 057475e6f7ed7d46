// pwl_table.cuh -- internal helpers around pwl_table: cell-count choice,
// shared-memory budgets of the streaming kernels and their launch shapes.
#pragma once

#include <algorithm>

#include "pwl_common.cuh"

namespace pwl {

int64_t choose_cells(int64_t N, float a, float b, float hmin, int64_t requested);

// Records (cells + reserved chain area) the forward kernel can stage in
// shared memory; chain records beyond the reserve are read from global memory.
inline int64_t eval_smem_records(const pwl_table_s* t)
{
    const int64_t cap = (int64_t)(device_info().smem_optin / sizeof(float4));
    return std::min<int64_t>(t->K + t->chain_reserve, cap);
}
inline size_t eval_smem_bytes(const pwl_table_s* t) { return sizeof(float4) * eval_smem_records(t); }

// Backward: records, N+2 reciprocal lengths and 2(N+2) FP32 accumulators.
inline size_t backward_fixed_smem(const pwl_table_s* t) { return 12 * (size_t)(t->N + 2); }
inline int64_t backward_smem_records(const pwl_table_s* t)
{
    const size_t optin = device_info().smem_optin;
    const size_t fixed = backward_fixed_smem(t);
    if (fixed + 16 * 64 > optin) return -1;  // does not fit: unsupported
    const int64_t cap = (int64_t)((optin - fixed) / sizeof(float4));
    return std::min<int64_t>(t->K + t->chain_reserve, cap);
}
inline size_t backward_smem_bytes(const pwl_table_s* t)
{
    const int64_t r = backward_smem_records(t);
    return r < 0 ? 0 : sizeof(float4) * (size_t)r + backward_fixed_smem(t);
}

// Persistent grid of a kernel: resident CTAs per SM (registers, shared
// memory, threads) times the SM count.  Sets the kernel's dynamic shared
// memory limit first, which the occupancy query takes into account.
template <typename Kern>
inline cudaError_t occupancy_grid(Kern kern, int threads, size_t smem, int* grid)
{
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem);
    if (e != cudaSuccess) return e;
    *grid = std::max(occ, 1) * device_info().sms;
    return cudaSuccess;
}

}  // namespace pwl
