// Batched segmented sort with packed tiles.
//
// Every segment of length L (2 <= L <= tile) belongs to size class
// k = ceil(log2 L), raised to at least m - gap (gap <= 10: a tile never holds
// more than 1024 segments; the autotuner picks the gap and the tile size).  A tile of 2^m positions holds 2^(m-k) segments of one
// class, each padded (virtually) to 2^k positions, and the tile engine runs
// phases 1..k of the network on it (Sections 3.1, 4.1, 4.2): those phases
// never mix positions of different 2^k blocks, so each segment is sorted on
// its own.  Binning happens on the device (classify, scan, scatter), so the
// whole batch is one asynchronous launch sequence; persistent CTAs take
// tiles from an atomic counter.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "engine.cuh"
#include "seg.h"
#include "tile_pass.cuh"

namespace bitonic {

namespace {

constexpr int kSegTileThreads = 256;

__device__ __forceinline__ int seg_class(int32_t len, int m, int gap)
{
    if (len < 2) return kSegClassSkip;
    if (len > (1 << m)) return kSegClassLarge;
    int k = 32 - __clz((uint32_t)(len - 1));  // ceil(log2 len)
    return k < m - gap ? m - gap : k;
}

__global__ void k_seg_classify(const int32_t* __restrict__ offs, int nseg, int m, int gap, uint8_t* __restrict__ cls,
                               SegPlan* plan, int* status, int debug_checks)
{
    __shared__ int hist[kSegClasses];
    for (int i = threadIdx.x; i < kSegClasses; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
        const int32_t len = offs[s + 1] - offs[s];
        if (len < 0 && debug_checks) atomicCAS(status, 0, 1);
        const int c = seg_class(len, m, gap);
        cls[s] = (uint8_t)c;
        atomicAdd(&hist[c], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSegClasses; i += blockDim.x)
        if (hist[i]) atomicAdd(&plan->hist[i], hist[i]);
}

// One thread: segment and tile prefix sums per class.
__global__ void k_seg_scan(SegPlan* plan, int m)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int segs = 0, tiles = 0;
    for (int c = 0; c < kSegClasses; ++c) {
        plan->seg_start[c] = segs;
        plan->tile_start[c] = tiles;
        plan->cursor[c] = 0;
        segs += plan->hist[c];
        if (c >= 1 && c <= m) tiles += (plan->hist[c] + (1 << (m - c)) - 1) >> (m - c);
    }
    plan->tile_start[kSegClasses] = tiles;
    plan->total_tiles = tiles;
}

__global__ void k_seg_scatter(const uint8_t* __restrict__ cls, int nseg, SegPlan* plan, int32_t* __restrict__ order)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nseg; s += gridDim.x * blockDim.x) {
        const int c = cls[s];
        order[plan->seg_start[c] + atomicAdd(&plan->cursor[c], 1)] = s;
    }
}

// Packed tile sort.  K = uint32_t (keys) or uint64_t (composite of key and
// position in its segment, for pairs).
template <typename K, int LOG_R, int LOG_T, int MINB>
__global__ void __launch_bounds__(1 << LOG_T, MINB)
k_seg_tiles(uint32_t* __restrict__ keys, uint32_t* __restrict__ vals, const int32_t* __restrict__ offs,
            const int32_t* __restrict__ order, const SegPlan* __restrict__ plan,
            const TileParamsBig* __restrict__ descs, int* counter)
{
    using T = Tile<K, false, LOG_R, LOG_T>;
    using Vec = typename T::Vec;
    constexpr int M = LOG_R + LOG_T;
    constexpr bool kPairs = sizeof(K) == 8;
    constexpr K kPad = KeyTraits<K>::kMax;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Vec* sm = reinterpret_cast<Vec*>(smem_raw);
    int32_t* s_start = reinterpret_cast<int32_t*>(smem_raw + (size_t(1) << M) * sizeof(K));
    int32_t* s_len = s_start + kSegMaxPerTile;
    // the tile's class descriptor, copied from global memory per tile
    TileParamsBig* s_desc = reinterpret_cast<TileParamsBig*>(s_len + kSegMaxPerTile);
    __shared__ int s_item;
    const uint32_t x = threadIdx.x;
    const int total = plan->total_tiles;
    for (;;) {
        if (x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int t = s_item;
        if (t >= total) return;
        int k = 1;
        while (t >= plan->tile_start[k + 1]) ++k;
        const int per_tile = 1 << (M - k);
        const int first = plan->seg_start[k] + ((t - plan->tile_start[k]) << (M - k));
        const int count = min(per_tile, plan->seg_start[k] + plan->hist[k] - first);
        for (int b = x; b < count; b += blockDim.x) {
            const int s = order[first + b];
            s_start[b] = offs[s];
            s_len[b] = offs[s + 1] - offs[s];
        }
        {  // header and rounds of class k's descriptor
            const TileParamsBig* D = descs + k;
            const int words = (int)((offsetof(TileParamsBig, rounds) + D->nrounds * sizeof(RoundDesc)) / 4);
            const uint32_t* src = reinterpret_cast<const uint32_t*>(D);
            uint32_t* dst = reinterpret_cast<uint32_t*>(s_desc);
            for (int w = (int)x; w < words; w += (int)blockDim.x) dst[w] = src[w];
        }
        __syncthreads();
        const TileParamsBig& P = *s_desc;
        const RoundDesc& r0 = P.rounds[0];
        const uint32_t mask = (1u << k) - 1u;
        T tl;
        // Load in round 0's layout, element by element (segments start
        // anywhere).  A vector's components are consecutive positions of one
        // segment (every layout vector lies above the vector bits, and k is
        // at least 3), so its segment is looked up once.
        {
            const uint32_t Lt = thread_local_index<LOG_T>(r0, x);
#pragma unroll
            for (int v = 0; v < T::NV; ++v) {
                uint32_t Lv = Lt;
#pragma unroll
                for (int j = 0; j < T::NREG; ++j)
                    if ((v >> j) & 1) Lv ^= r0.reg_loc[j];
                const int b = (int)(Lv >> k);
                const uint32_t w0 = Lv & mask;
                int32_t st = 0, len = 0;
                if (b < count) {
                    st = s_start[b];
                    len = s_len[b];
                }
#pragma unroll
                for (int c = 0; c < T::VEC; ++c) {
                    const uint32_t w = w0 + (uint32_t)c;
                    K val = kPad;
                    if ((int)w < len) {
                        const uint32_t key = keys[st + w];
                        if constexpr (kPairs) val = ((K)key << 32) | w;
                        else val = key;
                    }
                    tl.r[v * T::VEC + c] = val;
                }
            }
        }
        // straight-line round code from the catalog for 4-byte keys (as in the
        // tile passes), per-step dispatch for composites
        constexpr int kCat = sizeof(K) == 4 ? LOG_R : 0;
        steps_in_place<kCat, false>(tl.r, r0);
        const int nr = P.nrounds;
        for (int rd = 1; rd < nr; ++rd) {
            // the write goes to the slots this thread read last round (no barrier)
            tl.smem_write(sm, P.rounds[rd - 1], x);
            round_barrier(P.rounds[rd]);
            tl.smem_read(sm, P.rounds[rd], x);
            steps_in_place<kCat, false>(tl.r, P.rounds[rd]);
        }
        // Store in the last round's layout.
        {
            const RoundDesc& rl = P.rounds[nr - 1];
            const uint32_t Lt = thread_local_index<LOG_T>(rl, x);
            uint32_t gathered[kPairs ? T::R : 1];
            if constexpr (kPairs) {
                // Values are gathered by original position before any of this
                // segment's values are overwritten (the segment lives in this tile).
#pragma unroll
                for (int v = 0; v < T::NV; ++v) {
                    uint32_t Lv = Lt;
#pragma unroll
                    for (int j = 0; j < T::NREG; ++j)
                        if ((v >> j) & 1) Lv ^= rl.reg_loc[j];
                    const int b = (int)(Lv >> k);
                    const uint32_t w0 = Lv & mask;
                    int32_t st = 0, len = 0;
                    if (b < count) {
                        st = s_start[b];
                        len = s_len[b];
                    }
#pragma unroll
                    for (int c = 0; c < T::VEC; ++c)
                        if ((int)(w0 + (uint32_t)c) < len)
                            gathered[v * T::VEC + c] = vals[st + (uint32_t)tl.r[v * T::VEC + c]];
                }
                __syncthreads();
            }
#pragma unroll
            for (int v = 0; v < T::NV; ++v) {
                uint32_t Lv = Lt;
#pragma unroll
                for (int j = 0; j < T::NREG; ++j)
                    if ((v >> j) & 1) Lv ^= rl.reg_loc[j];
                const int b = (int)(Lv >> k);
                const uint32_t w0 = Lv & mask;
                int32_t st = 0, len = 0;
                if (b < count) {
                    st = s_start[b];
                    len = s_len[b];
                }
#pragma unroll
                for (int c = 0; c < T::VEC; ++c) {
                    const uint32_t w = w0 + (uint32_t)c;
                    if ((int)w < len) {
                        const K val = tl.r[v * T::VEC + c];
                        if constexpr (kPairs) {
                            keys[st + w] = (uint32_t)(val >> 32);
                            vals[st + w] = gathered[v * T::VEC + c];
                        } else {
                            keys[st + w] = val;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <typename K, int LOG_R, int LOG_T>
constexpr size_t seg_tile_smem()
{
    return (size_t(1) << (LOG_R + LOG_T)) * sizeof(K) + 2 * kSegMaxPerTile * sizeof(int32_t) +
           sizeof(TileParamsBig);
}

}  // namespace

cudaError_t seg_tiles_init_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_seg_tiles<uint32_t, 6, 8, kSegTileBlocksKeys>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)seg_tile_smem<uint32_t, 6, 8>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_seg_tiles<uint32_t, 6, 8, kSegTileBlocksKeys>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_seg_tiles<uint32_t, 5, 8, kSegTileBlocksKeys>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)seg_tile_smem<uint32_t, 5, 8>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_seg_tiles<uint64_t, 5, 8, kSegTileBlocksPairs>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)seg_tile_smem<uint64_t, 5, 8>());
    return e;
}

// Enqueues classify, scan, scatter and the packed tile sort.  ws must hold
// SegPlan, nseg class bytes and nseg order entries (seg_tiles_ws_bytes).
// Tiles of 2^m keys (keys: m = 14, 256 threads x 64, or 13, 256 x 32; pairs:
// 8K composites, m = 13); the smallest class is m - gap.
cudaError_t seg_tiles_launch(uint32_t* keys, uint32_t* vals, const int32_t* offs, int nseg, void* ws,
                             const TileParamsBig* class_descs, int m, int gap, int grid, int* status,
                             int debug_checks, cudaStream_t s)
{
    const bool pairs = vals != nullptr;
    if ((pairs && m != 13) || (!pairs && m != 13 && m != 14) || gap < 1 || gap > 10) return cudaErrorInvalidValue;
    SegPlan* plan = reinterpret_cast<SegPlan*>(ws);
    int32_t* order = reinterpret_cast<int32_t*>(plan + 1);
    uint8_t* cls = reinterpret_cast<uint8_t*>(order + nseg);
    cudaError_t e = cudaMemsetAsync(plan, 0, sizeof(SegPlan), s);
    if (e != cudaSuccess) return e;
    int cgrid = (nseg + 255) / 256;
    cgrid = cgrid < 1 ? 1 : (cgrid > 1024 ? 1024 : cgrid);
    k_seg_classify<<<cgrid, 256, 0, s>>>(offs, nseg, m, gap, cls, plan, status, debug_checks);
    k_seg_scan<<<1, 32, 0, s>>>(plan, m);
    k_seg_scatter<<<cgrid, 256, 0, s>>>(cls, nseg, plan, order);
    if (pairs)
        k_seg_tiles<uint64_t, 5, 8, kSegTileBlocksPairs><<<grid, kSegTileThreads, seg_tile_smem<uint64_t, 5, 8>(), s>>>(
            keys, vals, offs, order, plan, class_descs, &plan->tile_counter);
    else if (m == 14)
        k_seg_tiles<uint32_t, 6, 8, kSegTileBlocksKeys><<<grid, kSegTileThreads, seg_tile_smem<uint32_t, 6, 8>(), s>>>(
            keys, nullptr, offs, order, plan, class_descs, &plan->tile_counter);
    else
        k_seg_tiles<uint32_t, 5, 8, kSegTileBlocksKeys><<<grid, kSegTileThreads, seg_tile_smem<uint32_t, 5, 8>(), s>>>(
            keys, nullptr, offs, order, plan, class_descs, &plan->tile_counter);
    return cudaGetLastError();
}

size_t seg_tiles_ws_bytes(int nseg)
{
    return sizeof(SegPlan) + (size_t)nseg * (sizeof(int32_t) + 1) + 16;
}

}  // namespace bitonic
