// Key/value sort that allocates no device memory.
//
// bitonic_sort_pairs_u32 keeps its 64-bit (key, index) composites in a
// workspace it grows with cudaMalloc.  Some callers cannot let a library do
// that: applications whose memory manager owns all device memory and forbids
// allocations behind its back, and latency-critical paths where cudaMalloc's
// implicit synchronisation is not acceptable.  This entry point keeps the
// composites in a fixed array in the library's own device image instead.
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <mutex>

#include "bitonic.h"
#include "internal.h"
#include "kernel_cfg.h"

namespace bitonic {
namespace {

// Largest pair count the fixed array holds: 2^20 composites of 8 bytes
// (8 MiB), kept by every GPU that loads the library until the process exits.
constexpr size_t kNoAllocMaxPairs = size_t(1) << 20;

// The scratch array.  Host code may not use this name as an address; each
// device's address is looked up once with cudaGetSymbolAddress.
static __device__ __align__(256) uint64_t g_noalloc_comp[kNoAllocMaxPairs];

struct NoAllocDevice {
    bool ready = false;
    uint64_t* comp = nullptr;  // device address of g_noalloc_comp on this device
};

std::mutex g_na_mu;
std::map<int, NoAllocDevice> g_na_dev;
std::map<uint64_t, std::unique_ptr<Plan>> g_na_plans;  // composite-sort plans by N (host memory only)

bitonic_status na_fail(cudaError_t, const char*)
{
    cudaGetLastError();  // clear a sticky launch error
    return BITONIC_ERR_CUDA;
}

// Once per device, with that device current: find the array's device
// address and raise the tile kernels' shared-memory limit.  Neither call
// allocates memory.
bitonic_status na_setup(NoAllocDevice** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(e, "cudaGetDevice");
    NoAllocDevice& d = g_na_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_comp);
        if (e != cudaSuccess) return na_fail(e, "cudaGetSymbolAddress");
        e = init_tile_attributes();
        if (e != cudaSuccess) return na_fail(e, "cudaFuncSetAttribute");
        d.comp = static_cast<uint64_t*>(p);
        d.ready = true;
    }
    *out = &d;
    return BITONIC_OK;
}

const Plan* na_plan(uint64_t n)
{
    uint64_t N = 2;
    while (N < n) N <<= 1;
    auto it = g_na_plans.find(N);
    if (it == g_na_plans.end()) {
        auto p = std::make_unique<Plan>(make_plan(N, 8, Options{}));
        it = g_na_plans.emplace(N, std::move(p)).first;
    }
    return it->second.get();
}

}  // namespace
}  // namespace bitonic

using namespace bitonic;

extern "C" bitonic_status bitonic_sort_pairs_u32_noalloc(uint32_t* keys, uint32_t* vals, size_t n, int ascending,
                                                         bitonic_stream_t stream)
{
    if (n > kNoAllocMaxPairs) return BITONIC_ERR_UNSUPPORTED;  // more than the fixed array holds
    if (n <= 1) return BITONIC_OK;
    if (!keys || !vals || ((uintptr_t)keys & 3u) || ((uintptr_t)vals & 3u)) return BITONIC_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> g(g_na_mu);
    NoAllocDevice* d;
    bitonic_status st = na_setup(&d);
    if (st) return st;
    const Plan* pl = na_plan(n);
    if (!pl->ok) return BITONIC_ERR_UNSUPPORTED;
    for (const Launch& L : pl->launches)
        if (L.kind == KIND_STEP || !L.small) return BITONIC_ERR_UNSUPPORTED;
    const uint32_t nn = (uint32_t)n;
    const int desc = ascending ? 0 : 1;
    // Every composite the sort reads at positions < n is written by the pack
    // kernel first, and positions >= n are virtual: nothing needs clearing.
    cudaError_t e = launch_pairs_pack(d->comp, keys, nn, desc, s);
    if (e != cudaSuccess) return na_fail(e, "pack");
    for (const Launch& L : pl->launches) {
        const TileParamsBig& D = pl->descs[L.desc];
        uint32_t ntiles = L.grid;
        if (D.contiguous) {
            const uint64_t live = ((uint64_t)nn + (1u << D.m) - 1) >> D.m;
            if (live < ntiles) ntiles = (uint32_t)live;
        }
        e = launch_tile(pl->cfg, d->comp, 0, nn, &pl->small[L.desc], nullptr, ntiles, KeyMapHost{}, KeyMapHost{}, s);
        if (e != cudaSuccess) return na_fail(e, "tile pass");
    }
    e = launch_pairs_gather(d->comp, vals, nn, s);
    if (e != cudaSuccess) return na_fail(e, "gather");
    e = launch_pairs_unpack(d->comp, keys, vals, nn, desc, s);
    if (e != cudaSuccess) return na_fail(e, "unpack");
    return BITONIC_OK;
}
