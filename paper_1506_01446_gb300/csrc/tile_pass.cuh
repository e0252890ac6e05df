// Tile-pass kernel templates (Sections 4.1 and 4.2), instantiated per key
// type in tile_u32.cu and tile_u64.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.cuh"
#include "kernel_cfg.h"
#include "patterns.h"
#include "tma.cuh"

namespace bitonic {

// Steps of catalog pattern IDX, unrolled at compile time (straight-line code,
// so the register allocator can rename freely inside a round).
template <int LOG_R, int IDX, int S, bool DESC, typename K, int R>
__device__ __forceinline__ void pattern_steps(K (&r)[R])
{
    constexpr RoundPattern p = catalog_pattern(LOG_R, IDX);
    if constexpr (S < p.n) {
        constexpr int code = p.steps[S];
        net_step<code & 15, (code & kStepFlip) != 0, DESC>(r);
        pattern_steps<LOG_R, IDX, S + 1, DESC>(r);
    }
}

// Runs a round's steps on registers that stay in place (round 0 and the
// last round): a catalog pattern, else the per-step dispatcher.
template <int LOG_R, bool DESC, int I = 0, typename K, int R>
__device__ __forceinline__ void steps_in_place(K (&r)[R], const RoundDesc& rd)
{
    if constexpr (I < catalog_size(LOG_R)) {
        if (rd.pattern == I) {
            pattern_steps<LOG_R, I, 0, DESC>(r);
            return;
        }
        steps_in_place<LOG_R, DESC, I + 1>(r, rd);
    } else {
        run_round_steps<DESC>(r, rd);
    }
}

// A middle round: shared-memory read, steps, shared-memory write, with the
// registers local to the round.  The write goes back to the slots this
// thread has just read (the same layout), so it needs no barrier: no other
// thread reads or writes those slots in this round.
template <typename K, bool DESC, int LOG_R, int LOG_T, bool CATALOG, int I = 0>
__device__ __forceinline__ void middle_round(typename Tile<K, DESC, LOG_R, LOG_T>::Vec* sm, const RoundDesc& rd,
                                             uint32_t x)
{
    using T = Tile<K, DESC, LOG_R, LOG_T>;
    if constexpr (CATALOG && I < catalog_size(LOG_R)) {
        if (rd.pattern == I) {
            T u;
            u.smem_read(sm, rd, x);
            pattern_steps<LOG_R, I, 0, DESC>(u.r);
            u.smem_write(sm, rd, x);
            return;
        }
        middle_round<K, DESC, LOG_R, LOG_T, CATALOG, I + 1>(sm, rd, x);
    } else {
        T u;
        u.smem_read(sm, rd, x);
        run_round_steps<DESC>(u.r, rd);
        u.smem_write(sm, rd, x);
    }
}

// Orders the previous round's shared-memory writes before this round's
// reads: a warp barrier where the planner marked the transpose warp-local
// (every warp reads back exactly the slots it wrote), else a CTA barrier.
// The flag is the same for every thread of the CTA.
__device__ __forceinline__ void round_barrier(const RoundDesc& rd)
{
    if (rd.warp_local)
        __syncwarp();
    else
        __syncthreads();
}

// The rounds of one tile once round 0's keys are in t's registers: round 0's
// steps, then each later round's shared-memory transpose and steps (Section
// 4.1 between rounds, Section 4.2 within them).  Leaves the last round's
// keys in t's registers.
template <typename K, bool DESC, int LOG_R, int LOG_T, bool CATALOG, class PT>
__device__ __forceinline__ void run_tile_rounds(Tile<K, DESC, LOG_R, LOG_T>& t,
                                                typename Tile<K, DESC, LOG_R, LOG_T>::Vec* sm, const PT& P,
                                                uint32_t x)
{
    constexpr int kCat = CATALOG ? LOG_R : 0;  // catalog_size(0) == 0: per-step dispatch only
    const int nr = P.nrounds;
    steps_in_place<kCat, DESC>(t.r, P.rounds[0]);
    if (nr > 1) {
        t.smem_write(sm, P.rounds[0], x);
        for (int rd = 1; rd < nr - 1; ++rd) {
            round_barrier(P.rounds[rd]);
            middle_round<K, DESC, LOG_R, LOG_T, CATALOG>(sm, P.rounds[rd], x);
        }
        round_barrier(P.rounds[nr - 1]);
        t.smem_read(sm, P.rounds[nr - 1], x);
        steps_in_place<kCat, DESC>(t.r, P.rounds[nr - 1]);
    }
}

// One tile pass (Sections 4.1 and 4.2): load a tile of 2^m keys, run the
// rounds (register network steps, shared-memory transposes in between), store.
// Prefetches into L2 the rows of the tile `dist` CTAs ahead (the one a CTA
// starting about one resident wave later will load), with TMA bulk
// prefetches: no registers or shared memory are spent on it.  Tiles are
// numbered from cta0 (a launch may cover a range of a pass's tiles).
template <typename K, int LOG_T, class PT>
__device__ __forceinline__ void prefetch_tile_l2(const K* base, uint32_t lo, uint32_t hi, const PT& P, uint32_t dist,
                                                 uint32_t cta0)
{
    const uint32_t t = blockIdx.x + dist;
    if (!dist || t >= gridDim.x) return;
    const uint32_t g0 = cta_base(P, cta0 + t);
    const int c = P.row_log;
    const uint32_t row_len = 1u << c;
    const uint32_t nrows = 1u << (P.m - c);
    // rows longer than 32 KiB are prefetched in 32 KiB pieces
    const uint32_t piece = row_len > 8192u ? 8192u : row_len;
    const uint32_t pieces = row_len / piece;
    for (uint32_t i = threadIdx.x; i < nrows * pieces; i += (1u << LOG_T)) {
        const uint32_t r = i / pieces, q = i % pieces;
        uint32_t g = g0;
        for (int j = 0; j < P.m - c; ++j)
            if ((r >> j) & 1u) g ^= P.gvec[c + j];
        g += q * piece;
        if (g >= lo && g + piece <= hi) l2_prefetch_bulk(base + g, piece * (uint32_t)sizeof(K));
    }
}

template <typename K, bool DESC, int LOG_R, int LOG_T, bool CATALOG, class PT>
__device__ __forceinline__ void tile_pass(K* __restrict__ base, uint32_t lo, uint32_t hi, const PT& P,
                                          KeyMap<K> m_in, KeyMap<K> m_out, uint32_t pf_dist = 0, uint32_t cta0 = 0)
{
    using T = Tile<K, DESC, LOG_R, LOG_T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto* sm = reinterpret_cast<typename T::Vec*>(smem_raw);
    const uint32_t x = threadIdx.x;
    const uint32_t g0 = cta_base(P, cta0 + blockIdx.x);
    if (P.contiguous && g0 >= hi) return;  // the whole tile is tail padding
    const bool interior = (g0 & ~P.span_mask) >= lo && (g0 | P.span_mask) < hi;
    T t;
    if (interior)
        t.load_global_interior(base, P.io[0], g0, x, m_in);
    else
        t.load_global(base, lo, hi, P.io[0], g0, x, m_in);
    prefetch_tile_l2<K, LOG_T>(base, lo, hi, P, pf_dist, cta0);
    run_tile_rounds<K, DESC, LOG_R, LOG_T, CATALOG>(t, sm, P, x);
    if (interior)
        t.store_global_interior(base, P.io[1], g0, x, m_out);
    else
        t.store_global(base, lo, hi, P.io[1], g0, x, m_out);
}

// Descriptor passed by value: every thread reads it through the constant
// bank.  Real keys pass through m_in on load and m_out on store (identity
// maps except on a sort's first and last launch: the complement of a
// descending sort, the order-preserving maps of signed and float keys).  The round
// catalog (straight-line code per round shape) pays for its instruction
// footprint with 4-byte keys (2^28: 13.5 vs 14.7 ms on GB300) but not with
// 8-byte composites (2^26 pairs: 10.33 vs 10.22 ms), which use per-step
// dispatch.  CTA i of the launch runs tile cta0 + i of the pass.
template <typename K, int LOG_R, int LOG_T, int MINB>
__global__ void __launch_bounds__(1 << LOG_T, MINB)
k_tile(K* __restrict__ base, uint32_t lo, uint32_t hi, const __grid_constant__ TileParams P, KeyMap<K> m_in,
       KeyMap<K> m_out, uint32_t pf_dist, uint32_t cta0)
{
    tile_pass<K, false, LOG_R, LOG_T, sizeof(K) == 4>(base, lo, hi, P, m_in, m_out, pf_dist, cta0);
}

// Descriptor with more rounds than fit by value, read from global memory.
template <typename K, int LOG_R, int LOG_T, int MINB>
__global__ void __launch_bounds__(1 << LOG_T, MINB)
k_tile_big(K* __restrict__ base, uint32_t lo, uint32_t hi, const TileParamsBig* __restrict__ P, KeyMap<K> m_in,
           KeyMap<K> m_out, uint32_t cta0)
{
    tile_pass<K, false, LOG_R, LOG_T, false>(base, lo, hi, *P, m_in, m_out, 0, cta0);
}

// Launcher and attribute setup of one configuration.
template <typename K, int LR, int LT, int MB>
cudaError_t launch_tile_t(void* base, uint32_t lo, uint32_t hi, const TileParams* hP, const TileParamsBig* dP,
                          uint32_t grid, const KeyMapHost& mi, const KeyMapHost& mo, uint32_t pf_dist, uint32_t cta0,
                          cudaStream_t s)
{
    constexpr int kThreads = 1 << LT;
    constexpr size_t kSmem = (size_t(1) << (LR + LT)) * sizeof(K);
    const KeyMap<K> ki{(K)mi.a, (K)mi.b, (K)mi.s}, ko{(K)mo.a, (K)mo.b, (K)mo.s};
    if (hP)
        k_tile<K, LR, LT, MB><<<grid, kThreads, kSmem, s>>>((K*)base, lo, hi, *hP, ki, ko, pf_dist, cta0);
    else
        k_tile_big<K, LR, LT, MB><<<grid, kThreads, kSmem, s>>>((K*)base, lo, hi, dP, ki, ko, cta0);
    return cudaGetLastError();
}

template <typename K, int LR, int LT, int MB>
cudaError_t tile_occupancy_t(int* blocks)
{
    constexpr int kSmem = (int)((size_t(1) << (LR + LT)) * sizeof(K));
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_tile<K, LR, LT, MB>, 1 << LT, kSmem);
}

template <typename K, int LR, int LT, int MB>
cudaError_t tile_attr_t()
{
    constexpr int kSmem = (int)((size_t(1) << (LR + LT)) * sizeof(K));
    cudaError_t e =
        cudaFuncSetAttribute(k_tile<K, LR, LT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tile_big<K, LR, LT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    // Prefer the largest shared-memory carve-out so that every CTA the
    // registers allow can be resident.
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tile<K, LR, LT, MB>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}


}  // namespace bitonic
