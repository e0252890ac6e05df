// Segmented sort helpers: the batch statistics that size the pair workspace,
// and the key complement of the descending sorts.  (Segments longer than
// one tile run their multi-pass plans: seg_long.cu.)
#include <cuda_runtime.h>
#include <stdint.h>

#include "seg.h"

namespace bitonic {

namespace {

// Span of the offsets (first, last) and the longest segment, for planning.
__global__ void k_seg_stats(const int32_t* __restrict__ offs, int nseg, int* out)
{
    int mx = 0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x)
        mx = max(mx, offs[s + 1] - offs[s]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&out[2], mx);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[0] = offs[0];
        out[1] = offs[nseg];
    }
}

// Complements every key of the segments' span [offs[0], offs[nseg]): a
// descending segmented sort is the ascending sort of the complemented keys
// (Section 3.1 sorts either way; ties of pairs stay ordered by index).
__global__ void k_seg_complement(uint32_t* __restrict__ keys, const int32_t* __restrict__ offs, int nseg)
{
    int64_t lo = offs[0];
    const int64_t hi = offs[nseg];
    if (lo < 0) lo = 0;  // offsets are non-negative by contract
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += stride) keys[i] = ~keys[i];
}

}  // namespace

cudaError_t seg_init_attributes()
{
    cudaError_t e = seg_tiles_init_attributes();
    if (e == cudaSuccess) e = seg_long_init_attributes();
    return e;
}

cudaError_t seg_launch_complement(uint32_t* keys, const int32_t* offs, int nseg, int grid, cudaStream_t s)
{
    k_seg_complement<<<grid, 256, 0, s>>>(keys, offs, nseg);
    return cudaGetLastError();
}

cudaError_t seg_launch_stats(const int32_t* offs, int nseg, int* out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, 3 * sizeof(int), s);
    if (e != cudaSuccess) return e;
    int grid = (nseg + 255) / 256;
    if (grid > 1024) grid = 1024;
    if (grid < 1) grid = 1;
    k_seg_stats<<<grid, 256, 0, s>>>(offs, nseg, out);
    return cudaGetLastError();
}

}  // namespace bitonic
