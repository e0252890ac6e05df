// Fused pair-sort tile kernels.  A pair sort runs the network of Section 3.1
// on 64-bit composites (key' << 32) | index (key' = key, or ~key when
// descending), which orders equal keys by original index.  The first tile
// launch of the plan builds the composites while it loads the caller's keys;
// the last one splits them while it stores: keys back to the caller's array,
// original indices to the workspace, from which a streaming kernel gathers
// the values.  Every launch in between is the plain composite tile pass.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel_cfg.h"
#include "tile_pass.cuh"

namespace bitonic {

namespace {

constexpr uint64_t kCompPad = 0xFFFFFFFFFFFFFFFFull;  // virtual tail positions sort last

__device__ __forceinline__ uint64_t make_comp(uint32_t key, uint32_t flip, uint32_t idx)
{
    return ((uint64_t)(key ^ flip) << 32) | idx;
}

// Load of the first launch in its load round's layout: composites of the
// caller's keys for real positions [0, hi), pads beyond.  Each 16-byte
// register vector holds the composites of positions pos and pos + 1 (pos
// even).
template <int LOG_R, int LOG_T>
__device__ __forceinline__ void load_pairs(Tile<uint64_t, false, LOG_R, LOG_T>& t, const PairIo& pio, uint32_t hi,
                                           const IoDesc& io, uint32_t g0, uint32_t x)
{
    using T = Tile<uint64_t, false, LOG_R, LOG_T>;
    const uint32_t gt = g0 ^ io_thread_global<LOG_T>(io, x);
    uint32_t gr[T::NREG];
#pragma unroll
    for (int j = 0; j < T::NREG; ++j) gr[j] = io.reg_glob[j];
#pragma unroll
    for (int v = 0; v < T::NV; ++v) {
        const uint32_t pos = gt ^ reg_local_index<T::NREG>(gr, v);
        uint64_t* dst = t.r + 2 * v;
        if (pos + 2 <= hi) {
            uint32_t k0, k1;
            if (pio.aligned8) {
                const uint2 kk = *reinterpret_cast<const uint2*>(pio.keys_in + pos);
                k0 = kk.x;
                k1 = kk.y;
            } else {
                k0 = pio.keys_in[pos];
                k1 = pio.keys_in[pos + 1];
            }
            dst[0] = make_comp(k0, pio.flip, pos);
            dst[1] = make_comp(k1, pio.flip, pos + 1);
        } else {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const uint32_t p = pos + c;
                dst[c] = p < hi ? make_comp(pio.keys_in[p], pio.flip, p) : kCompPad;
            }
        }
    }
}

// Store of the last launch in its store round's layout: each composite's key
// to keys_out and its original index to idx_out (the values are gathered by
// a separate streaming kernel, which keeps the random reads off the tile
// kernel's critical path).
template <int LOG_R, int LOG_T>
__device__ __forceinline__ void store_pairs(const Tile<uint64_t, false, LOG_R, LOG_T>& t, const PairIo& pio,
                                            uint32_t hi, const IoDesc& io, uint32_t g0, uint32_t x)
{
    using T = Tile<uint64_t, false, LOG_R, LOG_T>;
    const uint32_t gt = g0 ^ io_thread_global<LOG_T>(io, x);
    uint32_t gr[T::NREG];
#pragma unroll
    for (int j = 0; j < T::NREG; ++j) gr[j] = io.reg_glob[j];
#pragma unroll
    for (int v = 0; v < T::NV; ++v) {
        const uint32_t pos = gt ^ reg_local_index<T::NREG>(gr, v);
        const uint64_t c0 = t.r[2 * v], c1 = t.r[2 * v + 1];
        const uint32_t k0 = (uint32_t)(c0 >> 32) ^ pio.flip, k1 = (uint32_t)(c1 >> 32) ^ pio.flip;
        if (pos + 2 <= hi) {
            *reinterpret_cast<uint2*>(pio.idx_out + pos) = make_uint2((uint32_t)c0, (uint32_t)c1);
            if (pio.aligned8) {
                *reinterpret_cast<uint2*>(pio.keys_out + pos) = make_uint2(k0, k1);
            } else {
                pio.keys_out[pos] = k0;
                pio.keys_out[pos + 1] = k1;
            }
        } else if (pos < hi) {  // one real position left (pos + 1 is a pad)
            pio.keys_out[pos] = k0;
            pio.idx_out[pos] = (uint32_t)c0;
        }
    }
}

}  // namespace

// MODE bit 0: the launch builds the composites on load (the plan's first
// launch); bit 1: it splits them on store (the last).  Tiles wholly past the
// last real position have nothing to do.
template <int LOG_R, int LOG_T, int MINB, int MODE>
__global__ void __launch_bounds__(1 << LOG_T, MINB)
k_tile_pairs(uint64_t* __restrict__ comp, uint32_t hi, const __grid_constant__ TileParams P, const PairIo pio,
             uint32_t pf_dist)
{
    using T = Tile<uint64_t, false, LOG_R, LOG_T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto* sm = reinterpret_cast<typename T::Vec*>(smem_raw);
    const uint32_t x = threadIdx.x;
    const uint32_t g0 = cta_base(P, blockIdx.x);
    if (P.contiguous && g0 >= hi) return;
    const bool interior = (g0 | P.span_mask) < hi;
    const KeyMap<uint64_t> ident{0, 0, 0};
    T t;
    if constexpr (MODE & 1) {
        load_pairs<LOG_R, LOG_T>(t, pio, hi, P.io[0], g0, x);
        // the caller's keys of the tile one resident wave ahead (composite
        // positions are key positions; bulk prefetches need 16-byte aligned
        // addresses, so only for a 16-byte aligned key array)
        if ((reinterpret_cast<uintptr_t>(pio.keys_in) & 15u) == 0)
            prefetch_tile_l2<uint32_t, LOG_T>(pio.keys_in, 0, hi, P, pf_dist, 0);
    } else {
        if (interior)
            t.load_global_interior(comp, P.io[0], g0, x, ident);
        else
            t.load_global(comp, 0, hi, P.io[0], g0, x, ident);
        prefetch_tile_l2<uint64_t, LOG_T>(comp, 0, hi, P, pf_dist, 0);
    }
    run_tile_rounds<uint64_t, false, LOG_R, LOG_T, false>(t, sm, P, x);
    if constexpr (MODE & 2) {
        store_pairs<LOG_R, LOG_T>(t, pio, hi, P.io[1], g0, x);
    } else {
        if (interior)
            t.store_global_interior(comp, P.io[1], g0, x, ident);
        else
            t.store_global(comp, 0, hi, P.io[1], g0, x, ident);
    }
}

template <int LR, int LT, int MB>
cudaError_t launch_pairs_t(int mode, uint64_t* comp, uint32_t hi, const TileParams* hP, uint32_t grid,
                           const PairIo& pio, uint32_t pf_dist, cudaStream_t s)
{
    constexpr int kThreads = 1 << LT;
    constexpr size_t kSmem = (size_t(1) << (LR + LT)) * sizeof(uint64_t);
    switch (mode) {
    case 1: k_tile_pairs<LR, LT, MB, 1><<<grid, kThreads, kSmem, s>>>(comp, hi, *hP, pio, pf_dist); break;
    case 2: k_tile_pairs<LR, LT, MB, 2><<<grid, kThreads, kSmem, s>>>(comp, hi, *hP, pio, pf_dist); break;
    case 3: k_tile_pairs<LR, LT, MB, 3><<<grid, kThreads, kSmem, s>>>(comp, hi, *hP, pio, pf_dist); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int LR, int LT, int MB>
cudaError_t pairs_attr_t()
{
    constexpr int kSmem = (int)((size_t(1) << (LR + LT)) * sizeof(uint64_t));
    cudaError_t e = cudaFuncSetAttribute(k_tile_pairs<LR, LT, MB, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tile_pairs<LR, LT, MB, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tile_pairs<LR, LT, MB, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    for (int m = 1; m <= 3 && e == cudaSuccess; ++m) {
        const void* f = m == 1 ? (const void*)k_tile_pairs<LR, LT, MB, 1>
                                : (m == 2 ? (const void*)k_tile_pairs<LR, LT, MB, 2>
                                          : (const void*)k_tile_pairs<LR, LT, MB, 3>);
        e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    }
    return e;
}

// The composite configurations of the optimized variant: 8K composites as
// 256 threads x 32, registers bounded for two CTAs per SM (id 4) or capped
// for three (id 8).
#define BITONIC_PAIR_CONFIGS(X) \
    X(4, 5, 8, 2)               \
    X(8, 5, 8, 3)

bool tile_pairs_supported(int cfg)
{
#define BITONIC_SUP(ID, LR, LT, MB) \
    if (cfg == ID) return true;
    BITONIC_PAIR_CONFIGS(BITONIC_SUP)
#undef BITONIC_SUP
    return false;
}

cudaError_t launch_tile_pairs(int cfg, int mode, uint64_t* comp, uint32_t hi, const TileParams* hP, uint32_t grid,
                              const PairIo& pio, uint32_t pf_dist, cudaStream_t s)
{
    if (!hP) return cudaErrorInvalidValue;
#define BITONIC_CASE(ID, LR, LT, MB) \
    case ID: return launch_pairs_t<LR, LT, MB>(mode, comp, hi, hP, grid, pio, pf_dist, s);
    switch (cfg) {
        BITONIC_PAIR_CONFIGS(BITONIC_CASE)
        default: return cudaErrorInvalidValue;
    }
#undef BITONIC_CASE
}

cudaError_t init_tile_pairs_attributes()
{
    cudaError_t e = cudaSuccess;
#define BITONIC_ATTR(ID, LR, LT, MB) \
    if (e == cudaSuccess) e = pairs_attr_t<LR, LT, MB>();
    BITONIC_PAIR_CONFIGS(BITONIC_ATTR)
#undef BITONIC_ATTR
    return e;
}

}  // namespace bitonic
