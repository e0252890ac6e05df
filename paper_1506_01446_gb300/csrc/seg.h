// Segmented-sort launchers (segmented.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bitonic {

constexpr uint32_t kSegSmemKeys = 16384;   // keys-only segments sorted in shared memory
constexpr uint32_t kSegSmemPairs = 8192;   // pair segments sorted in shared memory

cudaError_t seg_init_attributes();
cudaError_t seg_launch_keys(uint32_t* keys, const int32_t* offs, int nseg, int* counter, int* status,
                            int debug_checks, int grid, cudaStream_t s);
cudaError_t seg_launch_pairs(uint32_t* keys, uint32_t* vals, const int32_t* offs, int nseg, uint64_t* comp,
                             int32_t comp_base, int* counter, int* status, int debug_checks, int grid,
                             cudaStream_t s);
// out[0] = offsets[0], out[1] = offsets[nseg], out[2] = longest segment.
cudaError_t seg_launch_stats(const int32_t* offs, int nseg, int* out, cudaStream_t s);

}  // namespace bitonic
