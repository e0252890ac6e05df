// Kernels of the single-array sort: the tile-pass kernel (tile sort, global
// multi-stride pass and tile merge share it), the one-step kernel of the
// basic variant, and the pack / gather / unpack kernels of the pair sort.
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.cuh"
#include "internal.h"
#include "kernel_cfg.h"

namespace bitonic {

// One tile pass (Sections 4.1 and 4.2): load a tile of 2^m keys, run the
// rounds (register network steps, shared-memory transposes in between), store.
template <typename K, bool DESC, int LOG_R, int LOG_T, class PT>
__device__ __forceinline__ void tile_pass(K* __restrict__ base, uint32_t lo, uint32_t hi, const PT& P)
{
    using T = Tile<K, DESC, LOG_R, LOG_T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto* sm = reinterpret_cast<typename T::Vec*>(smem_raw);
    const uint32_t x = threadIdx.x;
    const uint32_t g0 = cta_base(P, blockIdx.x);
    if (P.contiguous && g0 >= hi) return;  // the whole tile is tail padding
    T t;
    const int nr = P.nrounds;
    t.load_global(base, lo, hi, P.io[0], g0, x);
    run_round_steps<DESC>(t.r, P.rounds[0]);
    for (int rd = 1; rd < nr; ++rd) {
        if (rd > 1) __syncthreads();
        t.smem_write(sm, P.rounds[rd - 1], x);
        __syncthreads();
        t.smem_read(sm, P.rounds[rd], x);
        run_round_steps<DESC>(t.r, P.rounds[rd]);
    }
    t.store_global(base, lo, hi, P.io[1], g0, x);
}

// Descriptor passed by value: every thread reads it through the constant bank.
template <typename K, bool DESC, int LOG_R, int LOG_T>
__global__ void __launch_bounds__(1 << LOG_T)
k_tile(K* __restrict__ base, uint32_t lo, uint32_t hi, const __grid_constant__ TileParams P)
{
    tile_pass<K, DESC, LOG_R, LOG_T>(base, lo, hi, P);
}

// Descriptor with more rounds than fit by value, read from global memory.
template <typename K, bool DESC, int LOG_R, int LOG_T>
__global__ void __launch_bounds__(1 << LOG_T)
k_tile_big(K* __restrict__ base, uint32_t lo, uint32_t hi, const TileParamsBig* __restrict__ P)
{
    tile_pass<K, DESC, LOG_R, LOG_T>(base, lo, hi, *P);
}

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

template <typename K, bool DESC, int LOG_R, int LOG_T>
cudaError_t launch_tile_t(K* base, uint32_t lo, uint32_t hi, const TileParams* hP, const TileParamsBig* dP,
                          uint32_t grid, cudaStream_t s)
{
    constexpr int kThreads = 1 << LOG_T;
    constexpr size_t kSmem = (size_t(1) << (LOG_R + LOG_T)) * sizeof(K);
    if (hP)
        k_tile<K, DESC, LOG_R, LOG_T><<<grid, kThreads, kSmem, s>>>(base, lo, hi, *hP);
    else
        k_tile_big<K, DESC, LOG_R, LOG_T><<<grid, kThreads, kSmem, s>>>(base, lo, hi, dP);
    return cudaGetLastError();
}

template <typename K, bool DESC>
cudaError_t launch_step_t(K* base, uint32_t lo, uint32_t hi, uint32_t N, int j, int flip, cudaStream_t s)
{
    const uint32_t npairs = N / 2;
    const uint32_t grid = (npairs + 255) / 256;
    k_step<K, DESC><<<grid, 256, 0, s>>>(base, lo, hi, npairs, j, flip);
    return cudaGetLastError();
}

}  // namespace

template <typename KT, int LR, int LT>
static cudaError_t launch_cfg(int desc, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                              const TileParamsBig* dP, uint32_t grid, cudaStream_t s)
{
    if constexpr (sizeof(KT) == 4) {
        return desc ? launch_tile_t<KT, true, LR, LT>((KT*)base, lo, hi, hP, dP, grid, s)
                    : launch_tile_t<KT, false, LR, LT>((KT*)base, lo, hi, hP, dP, grid, s);
    } else {
        return launch_tile_t<KT, false, LR, LT>((KT*)base, lo, hi, hP, dP, grid, s);
    }
}

// Launches one tile pass: hP (host copy, passed by value) when the
// descriptor fits, else dP (device copy of the big descriptor).
cudaError_t launch_tile(int cfg, int desc, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                        const TileParamsBig* dP, uint32_t grid, cudaStream_t s)
{
#define BITONIC_CFG_CASE(ID, KT, LR, LT) \
    case ID: return launch_cfg<KT, LR, LT>(desc, base, lo, hi, hP, dP, grid, s);
    switch (cfg) {
        BITONIC_TILE_CONFIGS(BITONIC_CFG_CASE)
        default: return cudaErrorInvalidValue;
    }
#undef BITONIC_CFG_CASE
}

template <typename K, bool DESC, int LR, int LT>
static cudaError_t set_attr_t()
{
    constexpr int kSmem = (int)((size_t(1) << (LR + LT)) * sizeof(K));
    cudaError_t e = cudaFuncSetAttribute(k_tile<K, DESC, LR, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tile_big<K, DESC, LR, LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    return e;
}

template <typename KT, int LR, int LT>
static cudaError_t set_attr_cfg()
{
    cudaError_t e = set_attr_t<KT, false, LR, LT>();
    if constexpr (sizeof(KT) == 4) {
        if (e == cudaSuccess) e = set_attr_t<KT, true, LR, LT>();
    }
    return e;
}

// Raises the dynamic shared-memory limit of every tile kernel on the current
// device (must run before any launch or graph capture on that device).
cudaError_t init_tile_attributes()
{
    cudaError_t e = cudaSuccess;
#define BITONIC_CFG_ATTR(ID, KT, LR, LT) \
    if (e == cudaSuccess) e = set_attr_cfg<KT, LR, LT>();
    BITONIC_TILE_CONFIGS(BITONIC_CFG_ATTR)
#undef BITONIC_CFG_ATTR
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

cudaError_t launch_pairs_pack(uint64_t* comp, const uint32_t* keys, uint32_t n, int desc, cudaStream_t s)
{
    k_pairs_pack<<<grid_for(n), 256, 0, s>>>(comp, keys, n, desc);
    return cudaGetLastError();
}

cudaError_t launch_pairs_gather(uint64_t* comp, const uint32_t* vals, uint32_t n, cudaStream_t s)
{
    k_pairs_gather<<<grid_for(n), 256, 0, s>>>(comp, vals, n);
    return cudaGetLastError();
}

cudaError_t launch_pairs_unpack(const uint64_t* comp, uint32_t* keys, uint32_t* vals, uint32_t n, int desc,
                                cudaStream_t s)
{
    k_pairs_unpack<<<grid_for(n), 256, 0, s>>>(comp, keys, vals, n, desc);
    return cudaGetLastError();
}

}  // namespace bitonic
