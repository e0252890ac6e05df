// Segmented sort, segments longer than one tile (keys only).
//
// A segment of L keys whose first key lies `front` keys past a 16-byte
// boundary is the sort of N = 2^k virtual positions (k = ceil(log2(front +
// L)) >= 14; k = 14, a single tile, when the packed tiles hold 8K keys) with its real
// keys in [front, front + L): the network of Section 3.1 split into the same
// launches as a plain sort of N keys (tile sort, multi-stride passes, tile
// merges; Sections 4.1 and 4.2), whose descriptors are built once per k.
// All of a batch's long segments run in one persistent launch: work items
// (pass p, segment, tile t) are numbered pass by pass and taken from an
// atomic counter, and a tile of pass p first waits until every tile of pass
// p - 1 of its segment is done (a per-segment counter of finished tiles).
// A CTA only waits for items that running CTAs took earlier, so the launch
// always makes progress; every wait is bounded and reports a timeout in the
// device status word instead of hanging.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "engine.cuh"
#include "seg.h"
#include "tile_pass.cuh"

namespace bitonic {

namespace {

constexpr int kLongThreads = 256;
constexpr int kLongLogR = 6;  // the 4-byte default tile: 256 threads x 64 keys
constexpr int kLongLogT = 8;
constexpr int kLongBlocks = 2;
constexpr int kLongM = kLongLogR + kLongLogT;
constexpr int kDevTimeoutCode = 2;  // device status word: a wait gave up
constexpr int kDevTooLongCode = 1;  // a segment longer than the library's maximum sort

__device__ __forceinline__ int ceil_log2_u64(uint64_t v)
{
    int k = 0;
    while ((uint64_t(1) << k) < v) ++k;
    return k;
}

// The batch's long segments: the packed-tile plan lists them (its large
// class) in `order`.
__device__ __forceinline__ void long_list(const SegPlan* plan, const int32_t* order, const int32_t** list, int* n)
{
    *list = order + plan->seg_start[kSegClassLarge];
    *n = plan->hist[kSegClassLarge];
}

// Keys between a segment's first key and the 16-byte boundary below it.
__device__ __forceinline__ uint32_t seg_front(const uint32_t* keys, int32_t start)
{
    return (uint32_t)(((uintptr_t)(keys + start) & 15u) >> 2);
}

__device__ __forceinline__ int long_class(const uint32_t* keys, const int32_t* offs, int s)
{
    const int32_t start = offs[s];
    const uint64_t v = (uint64_t)seg_front(keys, start) + (uint64_t)(offs[s + 1] - start);
    return ceil_log2_u64(v);
}

__global__ void k_long_classify(const uint32_t* keys, const int32_t* __restrict__ offs, const SegPlan* __restrict__ plan,
                                const int32_t* __restrict__ order, LongSched* sched, int* status)
{
    const int32_t* list;
    int n;
    long_list(plan, order, &list, &n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k = long_class(keys, offs, list[i]);
        if (k > 31) {
            atomicCAS(status, 0, kDevTooLongCode);
            continue;
        }
        atomicAdd(&sched->count[k], 1);
    }
}

// One thread: class slots (k descending, so that the classes still active
// in pass p are a prefix) and the first work item of every pass.
__global__ void k_long_scan(LongSched* sched, const LongPlans plans)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int m = plans.tile_log;
    int pos = 0;
    for (int k = 31; k >= m; --k) {
        sched->class_start[k] = pos;
        sched->cursor[k] = 0;
        pos += sched->count[k];
    }
    int items = 0;
    for (int p = 0; p < kLongMaxPasses; ++p) {
        sched->pass_start[p] = items;
        for (int k = 31; k >= m; --k)
            if (plans.npass[k] > p) items += sched->count[k] << (k - m);
    }
    sched->pass_start[kLongMaxPasses] = items;
    sched->total_items = items;
    sched->work = 0;
}

__global__ void k_long_scatter(const uint32_t* keys, const int32_t* __restrict__ offs, const SegPlan* __restrict__ plan,
                               const int32_t* __restrict__ order, LongSched* sched, int32_t* __restrict__ slots,
                               int32_t* __restrict__ done)
{
    const int32_t* list;
    int n;
    long_list(plan, order, &list, &n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = list[i];
        const int k = long_class(keys, offs, s);
        if (k > 31) continue;
        const int slot = sched->class_start[k] + atomicAdd(&sched->cursor[k], 1);
        slots[slot] = s;
        done[slot] = 0;
    }
}

// Bounded wait until *ctr >= need (thread 0 of the CTA); false if it gave up.
__device__ __forceinline__ bool wait_count(const int32_t* ctr, int need, uint32_t max_spins)
{
    for (uint32_t i = 0;; ++i) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= need) return true;
        if (i >= max_spins) return false;
        __nanosleep(128);
    }
}

// Shared memory: the tile, then the descriptor of the item's launch.
constexpr size_t kLongTileBytes = (size_t(1) << kLongM) * sizeof(uint32_t);
constexpr size_t kLongSmem = kLongTileBytes + sizeof(TileParamsBig);

__global__ void __launch_bounds__(kLongThreads, kLongBlocks)
k_long_sort(uint32_t* __restrict__ keys, const int32_t* __restrict__ offs, const int32_t* __restrict__ slots,
            int32_t* done, LongSched* sched, const LongPlans plans, const TileParamsBig* __restrict__ descs,
            int* status, uint32_t max_spins)
{
    using T = Tile<uint32_t, false, kLongLogR, kLongLogT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto* sm = reinterpret_cast<T::Vec*>(smem_raw);
    auto* P = reinterpret_cast<TileParamsBig*>(smem_raw + kLongTileBytes);
    __shared__ int s_item;
    const uint32_t x = threadIdx.x;
    const int m = plans.tile_log;
    const int total = sched->total_items;
    for (;;) {
        if (x == 0) s_item = atomicAdd(&sched->work, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) return;
        // item -> (pass p, class k, segment slot, tile t)
        int p = 0;
        while (item >= sched->pass_start[p + 1]) ++p;
        int o = item - sched->pass_start[p];
        int k = 31;
        for (; k >= m; --k) {
            if (plans.npass[k] <= p) continue;
            const int sz = sched->count[k] << (k - m);
            if (o < sz) break;
            o -= sz;
        }
        const int tl = k - m;
        const int slot = sched->class_start[k] + (o >> tl);
        const uint32_t t = (uint32_t)o & ((1u << tl) - 1u);
        const int s = slots[slot];
        const int32_t start = offs[s];
        const uint32_t front = seg_front(keys, start);
        const uint32_t hi = front + (uint32_t)(offs[s + 1] - start);
        uint32_t* base = keys + (start - (int32_t)front);
        // every tile of this segment's previous launch must be done
        if (x == 0 && p > 0 && !wait_count(done + slot, p << tl, max_spins)) atomicCAS(status, 0, kDevTimeoutCode);
        // the launch's descriptor (header and its rounds) into shared memory
        {
            const TileParamsBig* D = descs + plans.desc0[k] + p;
            const int words = (int)((offsetof(TileParamsBig, rounds) + D->nrounds * sizeof(RoundDesc)) / 4);
            const uint32_t* src = reinterpret_cast<const uint32_t*>(D);
            uint32_t* dst = reinterpret_cast<uint32_t*>(P);
            for (int w = (int)x; w < words; w += kLongThreads) dst[w] = src[w];
        }
        __threadfence();
        __syncthreads();
        const uint32_t g0 = cta_base(*P, t);
        if (!(P->contiguous && g0 >= hi)) {
            const bool interior = (g0 & ~P->span_mask) >= front && (g0 | P->span_mask) < hi;
            const KeyMap<uint32_t> ident{0u, 0u, 0u};
            T tile;
            if (interior)
                tile.load_global_interior<true>(base, P->io[0], g0, x, ident);
            else
                tile.load_global<true>(base, front, hi, P->io[0], g0, x, ident);
            run_tile_rounds<uint32_t, false, kLongLogR, kLongLogT, true>(tile, sm, *P, x);
            if (interior)
                tile.store_global_interior(base, P->io[1], g0, x, ident);
            else
                tile.store_global(base, front, hi, P->io[1], g0, x, ident);
        }
        __threadfence();
        __syncthreads();  // stores done; shared memory and s_item free for the next item
        if (x == 0) atomicAdd(done + slot, 1);
    }
}

}  // namespace

size_t seg_long_ws_offset(int nseg) { return (seg_tiles_ws_bytes(nseg) + 15) & ~size_t(15); }

size_t seg_long_ws_bytes(int nseg)
{
    return seg_long_ws_offset(nseg) + sizeof(LongSched) + 2 * (size_t)nseg * sizeof(int32_t) + 16;
}

cudaError_t seg_long_init_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_long_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLongSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_long_sort, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

cudaError_t seg_long_launch(uint32_t* keys, const int32_t* offs, int nseg, void* ws, const LongPlans& plans,
                            const TileParamsBig* descs, int grid, int* status, uint32_t max_spins, cudaStream_t s)
{
    if (plans.tile_log != kLongM) return cudaErrorInvalidValue;
    const SegPlan* plan = reinterpret_cast<const SegPlan*>(ws);
    const int32_t* order = reinterpret_cast<const int32_t*>(plan + 1);
    LongSched* sched = reinterpret_cast<LongSched*>(reinterpret_cast<char*>(ws) + seg_long_ws_offset(nseg));
    int32_t* slots = reinterpret_cast<int32_t*>(sched + 1);
    int32_t* done = slots + nseg;
    cudaError_t e = cudaMemsetAsync(sched, 0, sizeof(LongSched), s);
    if (e != cudaSuccess) return e;
    int cgrid = (nseg + 255) / 256;
    cgrid = cgrid < 1 ? 1 : (cgrid > 1024 ? 1024 : cgrid);
    k_long_classify<<<cgrid, 256, 0, s>>>(keys, offs, plan, order, sched, status);
    k_long_scan<<<1, 32, 0, s>>>(sched, plans);
    k_long_scatter<<<cgrid, 256, 0, s>>>(keys, offs, plan, order, sched, slots, done);
    k_long_sort<<<grid, kLongThreads, kLongSmem, s>>>(keys, offs, slots, done, sched, plans, descs, status, max_spins);
    return cudaGetLastError();
}

}  // namespace bitonic
