// Segmented sort of pairs: segments longer than one tile, and the batch
// statistics used to size the pair workspace.  Each long pair segment is
// sorted by one CTA running the network of Section 3.1 (mirror form) on
// global memory with block barriers between steps; persistent CTAs pull
// segments from an atomic counter.  (Long keys-only segments run their
// multi-pass plans instead: seg_long.cu.)
#include <cuda_runtime.h>
#include <stdint.h>

#include "seg.h"

namespace bitonic {

namespace {

constexpr int kSegThreads = 256;

__device__ __forceinline__ uint32_t next_pow2_u32(uint32_t v)
{
    uint32_t N = 1;
    while (N < v) N <<= 1;
    return N;
}

__device__ __forceinline__ int log2_u32(uint32_t N)
{
    return 31 - __clz(N);
}

// Same network on global memory with virtual padding (partner >= len is a
// no-op).  One CTA; __syncthreads orders its global accesses.
template <typename K>
__device__ void global_network(K* a, uint32_t len)
{
    const uint32_t N = next_pow2_u32(len);
    const int k = log2_u32(N);
    for (int p = 1; p <= k; ++p) {
        for (int j = p - 1; j >= 0; --j) {
            for (uint32_t q = threadIdx.x; q < N / 2; q += blockDim.x) {
                const uint32_t i = ((q >> j) << (j + 1)) | (q & ((1u << j) - 1u));
                const uint32_t pr = (j == p - 1) ? (i ^ ((2u << j) - 1u)) : (i | (1u << j));
                if (pr >= len) continue;
                const K x = a[i], y = a[pr];
                if (y < x) {
                    a[i] = y;
                    a[pr] = x;
                }
            }
            __syncthreads();
        }
    }
}

// Segments longer than one tile (the large class of a batch), one CTA each,
// taken from the batch's class-ordered list.  Pairs sort 64-bit composites
// (key, position) kept in comp at the segment's offset minus comp_base.
__global__ void __launch_bounds__(kSegThreads)
k_seg_large(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, const int32_t* __restrict__ offs,
            const int32_t* __restrict__ order, SegPlan* plan, uint64_t* __restrict__ comp, int32_t comp_base)
{
    __shared__ int item;
    const int n_large = plan->hist[kSegClassLarge];
    const int32_t* list = order + plan->seg_start[kSegClassLarge];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(&plan->large_counter, 1);
        __syncthreads();
        const int i = item;
        if (i >= n_large) return;
        const int s = list[i];
        const int32_t b = offs[s];
        const uint32_t len = (uint32_t)(offs[s + 1] - b);
        uint32_t* sk = keys + b;
        if (!vals) {
            global_network(sk, len);
            continue;
        }
        uint32_t* sv = vals + b;
        uint64_t* c = comp + (b - comp_base);
        for (uint32_t j = threadIdx.x; j < len; j += blockDim.x) c[j] = ((uint64_t)sk[j] << 32) | j;
        __syncthreads();
        global_network(c, len);
        for (uint32_t j = threadIdx.x; j < len; j += blockDim.x) c[j] = (c[j] & ~0xFFFFFFFFull) | sv[(uint32_t)c[j]];
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < len; j += blockDim.x) {
            sk[j] = (uint32_t)(c[j] >> 32);
            sv[j] = (uint32_t)c[j];
        }
    }
}

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

cudaError_t seg_launch_large(uint32_t* keys, uint32_t* vals, const int32_t* offs, void* ws, uint64_t* comp,
                             int32_t comp_base, int grid, cudaStream_t s)
{
    SegPlan* plan = reinterpret_cast<SegPlan*>(ws);
    const int32_t* order = reinterpret_cast<const int32_t*>(plan + 1);
    k_seg_large<<<grid, kSegThreads, 0, s>>>(keys, vals, offs, order, plan, comp, comp_base);
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
