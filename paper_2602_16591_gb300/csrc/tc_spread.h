// Tensor-core spreading (tc_spread.cu): float32 plans, tile edge 8, window support P in [3, 14].
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "device.cuh"

namespace pswf {

// accumulator row blocks of 128 (y, z) rows: ceil(E^2 / 128), E = 8 + P - 1
__host__ __device__ constexpr int tc_spread_mblocks(int P) { return ((7 + P) * (7 + P) + 127) / 128; }
// tensor-memory columns allocated per CTA (a power of two >= 32 x row blocks)
__host__ __device__ constexpr int tc_spread_tmem_cols(int P) {
    return tc_spread_mblocks(P) * 32 <= 32 ? 32 : (tc_spread_mblocks(P) * 32 <= 64 ? 64 : 128);
}

bool tc_spread_supports(int P);
size_t tc_spread_smem(int P, int degw);
// Spreading of one float32 plan into the tile slabs (same layout as k_spread); err_flag (device int,
// zeroed by the caller) is set when an MMA completion wait runs out.
cudaError_t launch_spread_tc(int P, int ntiles, const Vec4<float>* rec, const int2* idx, const int* tile_off,
                             const float* wcoef, int degw, SpreadChain ch, float* scratch, int* err_flag, cudaStream_t s);

// One warp waits (bounded by max_cycles SM clocks) on an mbarrier that nothing arrives at and sets
// *flag (device int) to 1 when the wait ran out.
cudaError_t launch_wait_probe(long long max_cycles, int* flag, cudaStream_t s);

}  // namespace pswf
