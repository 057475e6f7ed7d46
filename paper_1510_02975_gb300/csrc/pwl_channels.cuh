// pwl_channels.cuh -- internal interface of the channel-wise kernels.
#pragma once

#include "pwl_table.cuh"

namespace pwl {

struct ChanArgs {
    const float* knots;   // [C, N+1] FP32
    const float* values;  // [C, N+1] FP32
    int64_t C, R;         // channels, rows
    int N, K;             // intervals, cells per channel
    int64_t tiles, units, rows_per_unit, per_pair;
    int* status;          // device word: bit 0 set if a channel's knots are not strictly increasing
};

size_t channels_smem_bytes(int64_t N, int64_t K, bool backward);
int64_t channels_default_cells(int64_t N, bool backward);

}  // namespace pwl
