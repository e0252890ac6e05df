// Segmented sort: many independent arrays sorted ascending in one launch.
// CTAs pull segments from an atomic work counter (persistent kernel).  A
// segment that fits in shared memory is sorted there with the network of
// Section 3.1 in mirror form (Section 4.1: one CTA, block barriers between
// steps); longer segments run the same network on global memory, still one
// CTA per segment.
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

// Mirror-form network over N (power of two) entries of smem array a, all
// ascending.  Positions >= len already hold the maximal pad.
template <typename K>
__device__ void smem_network(K* a, uint32_t N)
{
    const int k = log2_u32(N);
    for (int p = 1; p <= k; ++p) {
        for (int j = p - 1; j >= 0; --j) {
            for (uint32_t q = threadIdx.x; q < N / 2; q += blockDim.x) {
                const uint32_t i = ((q >> j) << (j + 1)) | (q & ((1u << j) - 1u));
                const uint32_t pr = (j == p - 1) ? (i ^ ((2u << j) - 1u)) : (i | (1u << j));
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

__global__ void __launch_bounds__(kSegThreads)
k_seg_keys(uint32_t* __restrict__ keys, const int32_t* __restrict__ offs, int nseg, int* counter, int* status,
           int debug_checks)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t* a = reinterpret_cast<uint32_t*>(smem_raw);
    __shared__ int item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(counter, 1);
        __syncthreads();
        const int s = item;
        if (s >= nseg) return;
        const int32_t b = offs[s], e = offs[s + 1];
        if (e < b) {
            if (debug_checks && threadIdx.x == 0) atomicCAS(status, 0, 1);
            continue;
        }
        const uint32_t len = (uint32_t)(e - b);
        if (len < 2) continue;
        uint32_t* seg = keys + b;
        if (len <= kSegSmemKeys) {
            const uint32_t N = next_pow2_u32(len);
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) a[i] = i < len ? seg[i] : 0xFFFFFFFFu;
            __syncthreads();
            smem_network(a, N);
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) seg[i] = a[i];
        } else {
            global_network(seg, len);
        }
    }
}

__global__ void __launch_bounds__(kSegThreads)
k_seg_pairs(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, const int32_t* __restrict__ offs,
            int nseg, uint64_t* __restrict__ comp, int32_t comp_base, int* counter, int* status,
            int debug_checks)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t* a = reinterpret_cast<uint64_t*>(smem_raw);
    uint32_t* v = reinterpret_cast<uint32_t*>(a + kSegSmemPairs);
    __shared__ int item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(counter, 1);
        __syncthreads();
        const int s = item;
        if (s >= nseg) return;
        const int32_t b = offs[s], e = offs[s + 1];
        if (e < b) {
            if (debug_checks && threadIdx.x == 0) atomicCAS(status, 0, 1);
            continue;
        }
        const uint32_t len = (uint32_t)(e - b);
        if (len < 2) continue;
        uint32_t* sk = keys + b;
        uint32_t* sv = vals + b;
        if (len <= kSegSmemPairs) {
            const uint32_t N = next_pow2_u32(len);
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
                a[i] = i < len ? (((uint64_t)sk[i] << 32) | i) : ~0ull;
                if (i < len) v[i] = sv[i];
            }
            __syncthreads();
            smem_network(a, N);
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
                sk[i] = (uint32_t)(a[i] >> 32);
                sv[i] = v[(uint32_t)a[i]];
            }
        } else {
            uint64_t* c = comp + (b - comp_base);
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) c[i] = ((uint64_t)sk[i] << 32) | i;
            __syncthreads();
            global_network(c, len);
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) c[i] = (c[i] & ~0xFFFFFFFFull) | sv[(uint32_t)c[i]];
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
                sk[i] = (uint32_t)(c[i] >> 32);
                sv[i] = (uint32_t)c[i];
            }
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

}  // namespace

cudaError_t seg_init_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_seg_keys, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kSegSmemKeys * sizeof(uint32_t)));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_seg_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kSegSmemPairs * (sizeof(uint64_t) + sizeof(uint32_t))));
}

cudaError_t seg_launch_keys(uint32_t* keys, const int32_t* offs, int nseg, int* counter, int* status,
                            int debug_checks, int grid, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_seg_keys<<<grid, kSegThreads, kSegSmemKeys * sizeof(uint32_t), s>>>(keys, offs, nseg, counter, status,
                                                                         debug_checks);
    return cudaGetLastError();
}

cudaError_t seg_launch_pairs(uint32_t* keys, uint32_t* vals, const int32_t* offs, int nseg, uint64_t* comp,
                             int32_t comp_base, int* counter, int* status, int debug_checks, int grid,
                             cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_seg_pairs<<<grid, kSegThreads, kSegSmemPairs * (sizeof(uint64_t) + sizeof(uint32_t)), s>>>(
        keys, vals, offs, nseg, comp, comp_base, counter, status, debug_checks);
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
