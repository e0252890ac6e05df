// Segmented sort: segments longer than one packed tile.
//
// A segment of L keys whose first element lies `front` elements past a
// 16-byte boundary is the sort of N = 2^k virtual positions (k =
// ceil(log2(front + L)), at least the tile size) with its real elements in
// [front, front + L): the network of Section 3.1 split into the same
// launches as a plain sort of N keys (tile sort, multi-stride passes, tile
// merges; Sections 4.1 and 4.2), whose descriptors are built once per k.
// Key sorts run on the caller's keys.  Pair sorts run on 64-bit composites
// (key << 32) | index-in-segment in a workspace, with three more passes per
// segment: pack (build the composites), gather (read each value by the
// composite's index into its low half) and split (write keys and values
// back); equal keys keep their original order.
//
// All of a batch's long segments run in one persistent launch: work items
// (pass p, segment, tile t) are numbered pass by pass and taken from an
// atomic counter, and an item of pass p first waits until every tile of pass
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
constexpr int kLongBlocks = 2;
constexpr int kDevTimeoutCode = 2;  // device status word: a wait gave up
constexpr int kDevTooLongCode = 1;  // a segment longer than the library's maximum sort

// Tile shape of the long-segment kernels: 4-byte keys as 256 threads x 64
// (16K-key tiles), composites as 256 threads x 32 (8K composites).
template <typename K>
struct LongShape;
template <>
struct LongShape<uint32_t> {
    static constexpr int LOG_R = 6, LOG_T = 8;
};
template <>
struct LongShape<uint64_t> {
    static constexpr int LOG_R = 5, LOG_T = 8;
};

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

// The array a segment's tiles run on (elements of K), at its first element.
template <typename K>
__device__ __forceinline__ K* seg_array(const LongIo& io, int32_t start)
{
    if constexpr (sizeof(K) == 8)
        return reinterpret_cast<K*>(io.comp) + (start - io.comp_first);
    else
        return reinterpret_cast<K*>(io.keys) + start;
}

// Elements between a segment's first element and the 16-byte boundary below it.
template <typename K>
__device__ __forceinline__ uint32_t seg_front(const LongIo& io, int32_t start)
{
    return (uint32_t)(((uintptr_t)seg_array<K>(io, start) & 15u) / sizeof(K));
}

template <typename K>
__device__ __forceinline__ int long_class(const LongIo& io, const int32_t* offs, int s)
{
    const int32_t start = offs[s];
    const uint64_t v = (uint64_t)seg_front<K>(io, start) + (uint64_t)(offs[s + 1] - start);
    return ceil_log2_u64(v);
}

template <typename K>
__global__ void k_long_classify(const LongIo io, const int32_t* __restrict__ offs, const SegPlan* __restrict__ plan,
                                const int32_t* __restrict__ order, LongSched* sched, int* status)
{
    const int32_t* list;
    int n;
    long_list(plan, order, &list, &n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k = long_class<K>(io, offs, list[i]);
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

template <typename K>
__global__ void k_long_scatter(const LongIo io, const int32_t* __restrict__ offs, const SegPlan* __restrict__ plan,
                               const int32_t* __restrict__ order, LongSched* sched, int32_t* __restrict__ slots,
                               int32_t* __restrict__ done)
{
    const int32_t* list;
    int n;
    long_list(plan, order, &list, &n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = list[i];
        const int k = long_class<K>(io, offs, s);
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

template <typename K>
constexpr size_t long_tile_bytes()
{
    return (size_t(1) << (LongShape<K>::LOG_R + LongShape<K>::LOG_T)) * sizeof(K);
}

// Shared memory: the tile, then the descriptor of the item's launch.
template <typename K>
constexpr size_t long_smem()
{
    return long_tile_bytes<K>() + sizeof(TileParamsBig);
}

template <typename K>
__global__ void __launch_bounds__(kLongThreads, kLongBlocks)
k_long_sort(const LongIo io, const int32_t* __restrict__ offs, const int32_t* __restrict__ slots, int32_t* done,
            LongSched* sched, const LongPlans plans, const TileParamsBig* __restrict__ descs, int* status,
            uint32_t max_spins)
{
    constexpr int LOG_R = LongShape<K>::LOG_R, LOG_T = LongShape<K>::LOG_T;
    constexpr bool kPairs = sizeof(K) == 8;
    using T = Tile<K, false, LOG_R, LOG_T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto* sm = reinterpret_cast<typename T::Vec*>(smem_raw);
    auto* P = reinterpret_cast<TileParamsBig*>(smem_raw + long_tile_bytes<K>());
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
        const uint32_t len = (uint32_t)(offs[s + 1] - start);
        const uint32_t front = seg_front<K>(io, start);
        const uint32_t hi = front + len;
        K* base = seg_array<K>(io, start) - front;  // virtual position 0 of the segment's sort
        // every tile of this segment's previous pass must be done
        if (x == 0 && p > 0 && !wait_count(done + slot, p << tl, max_spins)) atomicCAS(status, 0, kDevTimeoutCode);
        const int np = plans.npass[k];
        // pair segments: pass 0 packs, the last two gather and split; the
        // plan's launches are passes 1 .. np - 3
        const int plan_pass = kPairs ? p - 1 : p;
        const bool plan_item = !kPairs || (p >= 1 && p <= np - 3);
        if (plan_item) {  // the launch's descriptor (header and its rounds) into shared memory
            const TileParamsBig* D = descs + plans.desc0[k] + plan_pass;
            const int words = (int)((offsetof(TileParamsBig, rounds) + D->nrounds * sizeof(RoundDesc)) / 4);
            const uint32_t* src = reinterpret_cast<const uint32_t*>(D);
            uint32_t* dst = reinterpret_cast<uint32_t*>(P);
            for (int w = (int)x; w < words; w += kLongThreads) dst[w] = src[w];
        }
        __threadfence();
        __syncthreads();
        if (plan_item) {
            const uint32_t g0 = cta_base(*P, t);
            if (!(P->contiguous && g0 >= hi)) {
                const bool interior = (g0 & ~P->span_mask) >= front && (g0 | P->span_mask) < hi;
                const KeyMap<K> ident{K(0), K(0), K(0)};
                T tile;
                if (interior)
                    tile.template load_global_interior<true>(base, P->io[0], g0, x, ident);
                else
                    tile.template load_global<true>(base, front, hi, P->io[0], g0, x, ident);
                run_tile_rounds<K, false, LOG_R, LOG_T, !kPairs>(tile, sm, *P, x);
                if (interior)
                    tile.store_global_interior(base, P->io[1], g0, x, ident);
                else
                    tile.store_global(base, front, hi, P->io[1], g0, x, ident);
            }
        } else if constexpr (kPairs) {
            // chunk t of the segment's virtual positions, real ones only
            const uint32_t q0 = max(t << m, front), q1 = min((t + 1) << m, hi);
            uint32_t* sk = io.keys + start;
            uint32_t* sv = io.vals + start;
            for (uint32_t q = q0 + x; q < q1; q += kLongThreads) {
                const uint32_t j = q - front;  // index in the segment
                if (p == 0) {
                    base[q] = ((uint64_t)sk[j] << 32) | j;
                } else if (p == np - 2) {  // values stay unchanged until the split pass
                    const uint64_t c = __ldcg(base + q);
                    base[q] = (c & 0xFFFFFFFF00000000ull) | sv[(uint32_t)c];
                } else {
                    const uint64_t c = __ldcg(base + q);
                    sk[j] = (uint32_t)(c >> 32);
                    sv[j] = (uint32_t)c;
                }
            }
        }
        __threadfence();
        __syncthreads();  // stores done; shared memory and s_item free for the next item
        if (x == 0) atomicAdd(done + slot, 1);
    }
}

template <typename K>
cudaError_t long_attr()
{
    cudaError_t e = cudaFuncSetAttribute(k_long_sort<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)long_smem<K>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_long_sort<K>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

template <typename K>
cudaError_t long_launch(const LongIo& io, const int32_t* offs, int nseg, void* ws, const LongPlans& plans,
                        const TileParamsBig* descs, int grid, int* status, uint32_t max_spins, cudaStream_t s)
{
    if (plans.tile_log != LongShape<K>::LOG_R + LongShape<K>::LOG_T) return cudaErrorInvalidValue;
    const SegPlan* plan = reinterpret_cast<const SegPlan*>(ws);
    const int32_t* order = reinterpret_cast<const int32_t*>(plan + 1);
    LongSched* sched = reinterpret_cast<LongSched*>(reinterpret_cast<char*>(ws) + seg_long_ws_offset(nseg));
    int32_t* slots = reinterpret_cast<int32_t*>(sched + 1);
    int32_t* done = slots + nseg;
    cudaError_t e = cudaMemsetAsync(sched, 0, sizeof(LongSched), s);
    if (e != cudaSuccess) return e;
    int cgrid = (nseg + 255) / 256;
    cgrid = cgrid < 1 ? 1 : (cgrid > 1024 ? 1024 : cgrid);
    k_long_classify<K><<<cgrid, 256, 0, s>>>(io, offs, plan, order, sched, status);
    k_long_scan<<<1, 32, 0, s>>>(sched, plans);
    k_long_scatter<K><<<cgrid, 256, 0, s>>>(io, offs, plan, order, sched, slots, done);
    k_long_sort<K><<<grid, kLongThreads, long_smem<K>(), s>>>(io, offs, slots, done, sched, plans, descs, status,
                                                             max_spins);
    return cudaGetLastError();
}

}  // namespace

size_t seg_long_ws_offset(int nseg) { return (seg_tiles_ws_bytes(nseg) + 15) & ~size_t(15); }

size_t seg_long_ws_bytes(int nseg)
{
    return seg_long_ws_offset(nseg) + sizeof(LongSched) + 2 * (size_t)nseg * sizeof(int32_t) + 16;
}

cudaError_t seg_long_init_attributes()
{
    cudaError_t e = long_attr<uint32_t>();
    if (e == cudaSuccess) e = long_attr<uint64_t>();
    return e;
}

cudaError_t seg_long_launch(const LongIo& io, const int32_t* offs, int nseg, void* ws, const LongPlans& plans,
                            const TileParamsBig* descs, int grid, int* status, uint32_t max_spins, cudaStream_t s)
{
    if (io.vals)
        return long_launch<uint64_t>(io, offs, nseg, ws, plans, descs, grid, status, max_spins, s);
    return long_launch<uint32_t>(io, offs, nseg, ws, plans, descs, grid, status, max_spins, s);
}

}  // namespace bitonic
