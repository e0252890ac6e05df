// Kernels of the single-array sort besides the tile passes: the one-step
// kernel of the basic variant and the pack / gather / unpack kernels of the
// pair sort; plus the dispatch of tile launches to their configuration.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "engine.cuh"
#include "kernel_cfg.h"

namespace bitonic {

// Section 3.3: one network step, one compare-exchange per thread.  Pair q of
// the step at stride bit j; FLIP steps pair i with i ^ (2^(j+1) - 1).
template <typename K, bool DESC>
__global__ void __launch_bounds__(256)
k_step(K* __restrict__ base, uint32_t lo, uint32_t hi, uint32_t npairs, int j, int flip)
{
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npairs) return;
    const uint32_t i = ((q >> j) << (j + 1)) | (q & ((1u << j) - 1u));
    const uint32_t p = flip ? (i ^ ((2u << j) - 1u)) : (i | (1u << j));
    // i < p.  A front pad at i or a tail pad at p makes the exchange a no-op.
    if (i < lo || p >= hi) return;
    const K a = base[i], b = base[p];
    if (DESC ? (a < b) : (b < a)) {
        base[i] = b;
        base[p] = a;
    }
}

// Pair sort, step 1: composite (key', index), key' = key or ~key.
__global__ void k_pairs_pack(uint64_t* __restrict__ comp, const uint32_t* __restrict__ keys, uint32_t n,
                             int desc)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t k = desc ? ~keys[i] : keys[i];
        comp[i] = ((uint64_t)k << 32) | i;
    }
}

// Pair sort, step 3: replace each composite's index by the value it names.
__global__ void k_pairs_gather(uint64_t* __restrict__ comp, const uint32_t* __restrict__ vals, uint32_t n)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t c = comp[i];
        comp[i] = (c & 0xFFFFFFFF00000000ull) | vals[(uint32_t)c];
    }
}

// Pair sort, step 4: split the composites back into keys and values.
__global__ void k_pairs_unpack(const uint64_t* __restrict__ comp, uint32_t* __restrict__ keys,
                               uint32_t* __restrict__ vals, uint32_t n, int desc)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t c = comp[i];
        const uint32_t k = (uint32_t)(c >> 32);
        keys[i] = desc ? ~k : k;
        vals[i] = (uint32_t)c;
    }
}

namespace {

template <typename K, bool DESC>
cudaError_t launch_step_t(K* base, uint32_t lo, uint32_t hi, uint32_t N, int j, int flip, cudaStream_t s)
{
    const uint32_t npairs = N / 2;
    const uint32_t grid = (npairs + 255) / 256;
    k_step<K, DESC><<<grid, 256, 0, s>>>(base, lo, hi, npairs, j, flip);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tile(int cfg, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                        const TileParamsBig* dP, uint32_t grid, const KeyMapHost& mi, const KeyMapHost& mo,
                        cudaStream_t s, uint32_t pf_dist, uint32_t cta0)
{
    if (tile_cfg(cfg).key_bytes == 4)
        return launch_tile_u32(cfg, base, lo, hi, hP, dP, grid, mi, mo, pf_dist, cta0, s);
    return launch_tile_u64(cfg, base, lo, hi, hP, dP, grid, mi, mo, pf_dist, cta0, s);
}

// One elementwise pass of a key map over base[lo, hi).
template <typename K>
__global__ void __launch_bounds__(256) k_keymap(K* __restrict__ base, uint32_t lo, uint32_t hi, KeyMap<K> m)
{
    for (uint32_t i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x)
        base[i] = m(base[i]);
}

cudaError_t launch_keymap(int key_bytes, void* base, uint32_t lo, uint32_t hi, const KeyMapHost& m, cudaStream_t s)
{
    if (hi <= lo) return cudaSuccess;
    uint32_t grid = (hi - lo + 255) / 256;
    if (grid > 4096) grid = 4096;
    if (key_bytes == 4)
        k_keymap<uint32_t><<<grid, 256, 0, s>>>((uint32_t*)base, lo, hi,
                                                KeyMap<uint32_t>{(uint32_t)m.a, (uint32_t)m.b, (uint32_t)m.s});
    else
        k_keymap<uint64_t><<<grid, 256, 0, s>>>((uint64_t*)base, lo, hi, KeyMap<uint64_t>{m.a, m.b, m.s});
    return cudaGetLastError();
}

// Resident CTAs per SM of a tile configuration (after init_tile_attributes).
cudaError_t tile_blocks_per_sm(int cfg, int* blocks)
{
    return tile_cfg(cfg).key_bytes == 4 ? tile_blocks_per_sm_u32(cfg, blocks) : tile_blocks_per_sm_u64(cfg, blocks);
}

// Raises the dynamic shared-memory limit of every tile kernel on the current
// device (must run before any launch or graph capture on that device).
cudaError_t init_tile_attributes()
{
    cudaError_t e = init_tile_attributes_u32();
    if (e == cudaSuccess) e = init_tile_attributes_u64();
    if (e == cudaSuccess) e = init_tile_pairs_attributes();
    return e;
}

cudaError_t launch_step(int key_bytes, int desc, void* base, uint32_t lo, uint32_t hi, uint32_t N, int j,
                        int flip, cudaStream_t s)
{
    if (key_bytes == 4)
        return desc ? launch_step_t<uint32_t, true>((uint32_t*)base, lo, hi, N, j, flip, s)
                    : launch_step_t<uint32_t, false>((uint32_t*)base, lo, hi, N, j, flip, s);
    return launch_step_t<uint64_t, false>((uint64_t*)base, lo, hi, N, j, flip, s);
}

static uint32_t grid_for(uint32_t n)
{
    uint32_t g = (n + 255) / 256;
    return g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g);
}

// Vector forms of the pair kernels: each thread moves groups of four
// elements as 16-byte vectors (composites as two 16-byte vectors), so that
// every SM keeps enough bytes in flight for HBM; the gather issues its four
// value reads independently.  Used when the key / value pointers are
// 16-byte aligned (the composite workspace always is); the tail of fewer
// than four elements is done element by element.
__global__ void __launch_bounds__(256) k_pairs_pack4(ulonglong2* __restrict__ comp, const uint4* __restrict__ keys,
                                                     uint32_t n4, uint32_t n, int desc)
{
    const uint32_t* keys1 = reinterpret_cast<const uint32_t*>(keys);  // element views for the tail
    uint64_t* comp1 = reinterpret_cast<uint64_t*>(comp);
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x) {
        uint4 k = keys[q];
        if (desc) {
            k.x = ~k.x; k.y = ~k.y; k.z = ~k.z; k.w = ~k.w;
        }
        const uint64_t i = 4ull * q;
        comp[2 * q] = make_ulonglong2(((uint64_t)k.x << 32) | i, ((uint64_t)k.y << 32) | (i + 1));
        comp[2 * q + 1] = make_ulonglong2(((uint64_t)k.z << 32) | (i + 2), ((uint64_t)k.w << 32) | (i + 3));
    }
    if (blockIdx.x == 0)
        for (uint32_t i = 4 * n4 + threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t k = desc ? ~keys1[i] : keys1[i];
            comp1[i] = ((uint64_t)k << 32) | i;
        }
}

__global__ void __launch_bounds__(256) k_pairs_gather4(ulonglong2* __restrict__ comp, const uint32_t* __restrict__ vals,
                                                       uint32_t n4, uint32_t n)
{
    uint64_t* comp1 = reinterpret_cast<uint64_t*>(comp);  // element view for the tail
    constexpr uint64_t kHi = 0xFFFFFFFF00000000ull;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x) {
        ulonglong2 a = comp[2 * q], b = comp[2 * q + 1];
        const uint32_t v0 = vals[(uint32_t)a.x], v1 = vals[(uint32_t)a.y];
        const uint32_t v2 = vals[(uint32_t)b.x], v3 = vals[(uint32_t)b.y];
        a.x = (a.x & kHi) | v0; a.y = (a.y & kHi) | v1;
        b.x = (b.x & kHi) | v2; b.y = (b.y & kHi) | v3;
        comp[2 * q] = a;
        comp[2 * q + 1] = b;
    }
    if (blockIdx.x == 0)
        for (uint32_t i = 4 * n4 + threadIdx.x; i < n; i += blockDim.x) {
            const uint64_t c = comp1[i];
            comp1[i] = (c & kHi) | vals[(uint32_t)c];
        }
}

__global__ void __launch_bounds__(256) k_pairs_unpack4(const ulonglong2* __restrict__ comp, uint4* __restrict__ keys,
                                                       uint4* __restrict__ vals, uint32_t n4, uint32_t n, int desc)
{
    const uint64_t* comp1 = reinterpret_cast<const uint64_t*>(comp);  // element views for the tail
    uint32_t* keys1 = reinterpret_cast<uint32_t*>(keys);
    uint32_t* vals1 = reinterpret_cast<uint32_t*>(vals);
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x) {
        const ulonglong2 a = comp[2 * q], b = comp[2 * q + 1];
        uint4 k = make_uint4((uint32_t)(a.x >> 32), (uint32_t)(a.y >> 32), (uint32_t)(b.x >> 32), (uint32_t)(b.y >> 32));
        if (desc) {
            k.x = ~k.x; k.y = ~k.y; k.z = ~k.z; k.w = ~k.w;
        }
        keys[q] = k;
        vals[q] = make_uint4((uint32_t)a.x, (uint32_t)a.y, (uint32_t)b.x, (uint32_t)b.y);
    }
    if (blockIdx.x == 0)
        for (uint32_t i = 4 * n4 + threadIdx.x; i < n; i += blockDim.x) {
            const uint64_t c = comp1[i];
            const uint32_t k = (uint32_t)(c >> 32);
            keys1[i] = desc ? ~k : k;
            vals1[i] = (uint32_t)c;
        }
}

// out[i] = vals[idx[i]]: four indices per thread as one 16-byte vector, the
// four value reads issued independently, the results written as one vector.
__global__ void __launch_bounds__(256) k_gather_by_index4(uint4* __restrict__ out, const uint32_t* __restrict__ vals,
                                                          const uint4* __restrict__ idx, uint32_t n4, uint32_t n)
{
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x) {
        const uint4 i = idx[q];
        out[q] = make_uint4(vals[i.x], vals[i.y], vals[i.z], vals[i.w]);
    }
    if (blockIdx.x == 0) {
        const uint32_t* idx1 = reinterpret_cast<const uint32_t*>(idx);
        uint32_t* out1 = reinterpret_cast<uint32_t*>(out);
        for (uint32_t i = 4 * n4 + threadIdx.x; i < n; i += blockDim.x) out1[i] = vals[idx1[i]];
    }
}

// One sweep of the sliced gather: lanes whose index lies in [lo, hi) read
// their value; the others keep what out holds from earlier sweeps (the
// first sweep writes 0 there, to be overwritten; a vector with no lane in
// the slice is not written at all).  The index and output streams are read
// and written with evict-first hints, so that the slice of vals, read at
// random, stays in L2 for the whole sweep.
__global__ void __launch_bounds__(256) k_gather_by_index_slice4(uint4* __restrict__ out,
                                                                const uint32_t* __restrict__ vals,
                                                                const uint4* __restrict__ idx, uint32_t n4,
                                                                uint32_t n, uint32_t lo, uint32_t hi, int first)
{
    const uint32_t w = hi - lo;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x) {
        const uint4 i = __ldcs(idx + q);
        const bool mx = i.x - lo < w, my = i.y - lo < w, mz = i.z - lo < w, mw = i.w - lo < w;
        if (!(mx || my || mz || mw)) continue;  // nothing of this slice: out stays as it is
        uint4 v = first ? make_uint4(0u, 0u, 0u, 0u) : __ldcs(out + q);
        if (mx) v.x = vals[i.x];
        if (my) v.y = vals[i.y];
        if (mz) v.z = vals[i.z];
        if (mw) v.w = vals[i.w];
        __stcs(out + q, v);
    }
    if (blockIdx.x == 0) {
        const uint32_t* idx1 = reinterpret_cast<const uint32_t*>(idx);
        uint32_t* out1 = reinterpret_cast<uint32_t*>(out);
        for (uint32_t i = 4 * n4 + threadIdx.x; i < n; i += blockDim.x) {
            const uint32_t j = idx1[i];
            if (j - lo < w) out1[i] = vals[j];
            else if (first) out1[i] = 0u;
        }
    }
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Values per slice of the sliced gather, in MiB of values (0: one plain
// sweep at every size).  Random 4-byte reads over a value array larger than
// L2 cost a DRAM sector each; in slices of 64 MiB they hit L2 after the
// first touch, for the price of reading the indices and rewriting the
// output once per slice: the gather of 2^26 values takes about 0.34 ms less
// in four slices (0.31 ms less in three, 0.25 in two, 0.05 in eight; 16
// slices are 0.9 ms slower).
#ifndef BITONIC_GATHER_SLICE_MB
#define BITONIC_GATHER_SLICE_MB 64
#endif
static constexpr uint64_t kGatherSliceKeys = (uint64_t)BITONIC_GATHER_SLICE_MB << 18;

int gather_launches(uint32_t n)
{
    if (kGatherSliceKeys == 0 || n <= kGatherSliceKeys) return 1;
    return (int)((n + kGatherSliceKeys - 1) / kGatherSliceKeys);
}

cudaError_t launch_gather_by_index(uint32_t* out, const uint32_t* vals, const uint32_t* idx, uint32_t n,
                                   cudaStream_t s)
{
    if (!aligned16(out) || !aligned16(idx)) return cudaErrorInvalidValue;
    const uint32_t n4 = n / 4;
    const int S = gather_launches(n);
    if (S == 1) {
        k_gather_by_index4<<<grid_for(n4 ? n4 : 1), 256, 0, s>>>((uint4*)out, vals, (const uint4*)idx, n4, n);
        return cudaGetLastError();
    }
    for (int k = 0; k < S; ++k) {
        const uint32_t lo = (uint32_t)((uint64_t)n * k / S), hi = (uint32_t)((uint64_t)n * (k + 1) / S);
        k_gather_by_index_slice4<<<grid_for(n4 ? n4 : 1), 256, 0, s>>>((uint4*)out, vals, (const uint4*)idx, n4, n,
                                                                       lo, hi, k == 0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pairs_pack(uint64_t* comp, const uint32_t* keys, uint32_t n, int desc, cudaStream_t s)
{
    if (aligned16(keys) && aligned16(comp)) {
        const uint32_t n4 = n / 4;
        k_pairs_pack4<<<grid_for(n4), 256, 0, s>>>((ulonglong2*)comp, (const uint4*)keys, n4, n, desc);
    } else {
        k_pairs_pack<<<grid_for(n), 256, 0, s>>>(comp, keys, n, desc);
    }
    return cudaGetLastError();
}

cudaError_t launch_pairs_gather(uint64_t* comp, const uint32_t* vals, uint32_t n, cudaStream_t s)
{
    if (aligned16(comp)) {
        const uint32_t n4 = n / 4;
        k_pairs_gather4<<<grid_for(n4), 256, 0, s>>>((ulonglong2*)comp, vals, n4, n);
    } else {
        k_pairs_gather<<<grid_for(n), 256, 0, s>>>(comp, vals, n);
    }
    return cudaGetLastError();
}

cudaError_t launch_pairs_unpack(const uint64_t* comp, uint32_t* keys, uint32_t* vals, uint32_t n, int desc,
                                cudaStream_t s)
{
    if (aligned16(comp) && aligned16(keys) && aligned16(vals)) {
        const uint32_t n4 = n / 4;
        k_pairs_unpack4<<<grid_for(n4), 256, 0, s>>>((const ulonglong2*)comp, (uint4*)keys, (uint4*)vals, n4, n,
                                                     desc);
    } else {
        k_pairs_unpack<<<grid_for(n), 256, 0, s>>>(comp, keys, vals, n, desc);
    }
    return cudaGetLastError();
}

}  // namespace bitonic
