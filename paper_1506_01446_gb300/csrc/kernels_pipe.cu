// Persistent, software-pipelined tile pass.  Each CTA walks its share of the
// tiles; while it runs the register network on tile i (Section 4.2) and the
// shared-memory transposes between rounds (Section 4.1), the rows of tile
// i + grid are already in flight: TMA bulk copies (cp.async.bulk) land them
// in a second shared-memory buffer and complete on an mbarrier.  Results go
// from registers straight to global memory in the store round's coalesced
// layout.
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.cuh"
#include "tile_pass.cuh"
#include "kernel_cfg.h"
#include "tma.cuh"

namespace bitonic {

namespace {

// Bound of each mbarrier wait (tries), and the copy-starving test mode: when
// set, each CTA arms its barrier for its first tile's bulk copies but issues
// none of them, so its first wait runs out with no copy in flight and the
// kernel reports a timeout (bitonic_debug_set_wait).
__device__ uint32_t g_pipe_wait_spins = kMaxWaitSpins;
__device__ int g_pipe_starve = 0;

// Shared memory: [landing tile][transpose tile][mbarrier][fill count][fill rows].
template <typename K, int M>
struct PipeSmem {
    static constexpr size_t kTileBytes = (size_t(1) << M) * sizeof(K);
    static constexpr int kMaxRows = 1 << (M - (sizeof(K) == 4 ? 5 : 4));
    static constexpr size_t kBarOff = 2 * kTileBytes;
    static constexpr size_t kCountOff = kBarOff + 8;
    static constexpr size_t kRowsOff = kCountOff + 8;
    static constexpr size_t kBytes = kRowsOff + 2 * kMaxRows;
};

template <class PT>
__device__ __forceinline__ uint32_t row_global(const PT& P, int c, uint32_t r)
{
    uint32_t g = 0;
    const int nb = P.m - c;
    for (int j = 0; j < nb; ++j)
        if ((r >> j) & 1u) g ^= P.gvec[c + j];
    return g;
}

template <int ASYNC, bool CATALOG, typename K, bool DESC, int LOG_R, int LOG_T, class PT>
__device__ __forceinline__ void pipe_pass(K* __restrict__ base, uint32_t lo, uint32_t hi, const PT& P,
                                          uint32_t ntiles, K cm_in, K cm_out, int* status)
{
    using T = Tile<K, DESC, LOG_R, LOG_T>;
    using Vec = typename T::Vec;
    using SM = PipeSmem<K, LOG_R + LOG_T>;
    constexpr uint32_t kThreads = 1u << LOG_T;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    K* X = reinterpret_cast<K*>(smem_raw);
    Vec* Y = reinterpret_cast<Vec*>(smem_raw + SM::kTileBytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + SM::kBarOff);
    uint32_t* fill_count = reinterpret_cast<uint32_t*>(smem_raw + SM::kCountOff);
    uint16_t* fill_rows = reinterpret_cast<uint16_t*>(smem_raw + SM::kRowsOff);

    const uint32_t x = threadIdx.x;
    const int c = P.row_log;
    const uint32_t row_len = 1u << c;
    const uint32_t nrows = 1u << (P.m - c);
    constexpr K kFront = T::kFrontPad, kTail = T::kTailPad;

    uint32_t tile = blockIdx.x;
    if (tile >= ntiles) return;
    if (x == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
        *fill_count = 0;
    }
    __syncthreads();

    // Rows of `t` that lie wholly in [lo, hi) go by TMA; the others are
    // listed for the CTA to fill (with pads where outside) after the next
    // barrier.  The copies may complete before the byte count is announced:
    // the barrier's transaction count goes below zero until thread 0's
    // arrive.expect_tx adds the total, and the phase cannot complete before
    // that arrival.
    const uint32_t max_spins = g_pipe_wait_spins;
    const bool starve = g_pipe_starve != 0;
    auto issue_tma = [&](uint32_t t) {
        const uint32_t g0 = cta_base(P, t);
        const bool skip = starve && t == blockIdx.x;  // test mode: the first tile's copies never start
        fence_proxy_async_smem();
        for (uint32_t r = x; r < nrows; r += kThreads) {
            const uint32_t g = g0 ^ row_global(P, c, r);
            if (g >= lo && g + row_len <= hi) {
                if (!skip) tma_load_bulk(X + (size_t)r * row_len, base + g, row_len * (uint32_t)sizeof(K), bar);
            } else
                fill_rows[atomicAdd(fill_count, 1u)] = (uint16_t)r;
        }
        __syncthreads();
        const uint32_t nfill = *fill_count;
        if (x == 0) mbar_arrive_expect_tx(bar, (nrows - nfill) * row_len * (uint32_t)sizeof(K));
        for (uint32_t i = x; i < nfill * row_len; i += kThreads) {
            const uint32_t r = fill_rows[i >> c];
            const uint32_t g = (g0 ^ row_global(P, c, r)) + (i & (row_len - 1));
            // pads are stored pre-complemented: the round-0 read complements every key
            X[(size_t)r * row_len + (i & (row_len - 1))] =
                g < lo ? (K)(kFront ^ cm_in) : (g >= hi ? (K)(kTail ^ cm_in) : base[g]);
        }
    };

    // The same prefetch with per-thread 16-byte cp.async copies in the load
    // round's coalesced layout (linear by local index in X).
    auto issue_cpasync = [&](uint32_t t) {
        const uint32_t g0 = cta_base(P, t);
        const RoundDesc& rd = P.rounds[0];
        const IoDesc& io = P.io[0];
        const uint32_t Lt = thread_local_index<LOG_T>(rd, x);
        const uint32_t gt = g0 ^ io_thread_global<LOG_T>(io, x);
#pragma unroll
        for (int v = 0; v < T::NV; ++v) {
            uint32_t L = Lt, g = gt;
#pragma unroll
            for (int j = 0; j < T::NREG; ++j)
                if ((v >> j) & 1) {
                    L ^= rd.reg_loc[j];
                    g ^= io.reg_glob[j];
                }
            K* dst = X + L;
            if (g >= lo && g + T::VEC <= hi) {
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(base + g)
                             : "memory");
            } else {
#pragma unroll
                for (int c2 = 0; c2 < T::VEC; ++c2) {
                    const uint32_t p = g + c2;
                    dst[c2] = p < lo ? (K)(kFront ^ cm_in) : (p >= hi ? (K)(kTail ^ cm_in) : base[p]);
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto issue = [&](uint32_t t) {
        if constexpr (ASYNC == 0) issue_tma(t);
        else issue_cpasync(t);
    };

    issue(tile);
    uint32_t parity = 0;
    T t;
    for (; tile < ntiles; tile += gridDim.x) {
        bool ok = true;
        if constexpr (ASYNC == 0) {
            ok = mbar_wait_bounded(bar, parity, max_spins);
            parity ^= 1u;
        } else {
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        __syncthreads();  // fill writes of this tile are complete
        t.smem_read_linear(reinterpret_cast<const Vec*>(X), P.rounds[0], x, cm_in);
        if (__syncthreads_or(!ok)) {
            if (x == 0) atomicCAS(status, 0, kStatusTimeout);
            if constexpr (ASYNC == 0) mbar_wait_bounded(bar, parity ^ 1u, max_spins);  // one more bounded wait for copies
            return;
        }
        const uint32_t g0 = cta_base(P, tile);
        const uint32_t next = tile + gridDim.x;
        if (x == 0) *fill_count = 0;
        __syncthreads();
        if (next < ntiles) issue(next);
        run_tile_rounds<K, DESC, LOG_R, LOG_T, CATALOG>(t, Y, P, x);
        t.store_global(base, lo, hi, P.io[1], g0, x, KeyMap<K>{K(0), cm_out, K(0)});
        __syncthreads();
    }
}

template <int ASYNC, typename K, int LOG_R, int LOG_T>
__global__ void __launch_bounds__(1 << LOG_T)
k_pipe(K* __restrict__ base, uint32_t lo, uint32_t hi, const __grid_constant__ TileParams P, uint32_t ntiles,
       K cm_in, K cm_out, int* status)
{
    pipe_pass<ASYNC, false, K, false, LOG_R, LOG_T>(base, lo, hi, P, ntiles, cm_in, cm_out, status);
}

template <int ASYNC, typename K, int LOG_R, int LOG_T>
__global__ void __launch_bounds__(1 << LOG_T)
k_pipe_big(K* __restrict__ base, uint32_t lo, uint32_t hi, const TileParamsBig* __restrict__ P, uint32_t ntiles,
           K cm_in, K cm_out, int* status)
{
    pipe_pass<ASYNC, false, K, false, LOG_R, LOG_T>(base, lo, hi, *P, ntiles, cm_in, cm_out, status);
}

template <typename K, int LR, int LT>
cudaError_t launch_pipe_t(int mode, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                          const TileParamsBig* dP, uint32_t ntiles, uint32_t grid, uint64_t xor_in,
                          uint64_t xor_out, int* status, cudaStream_t s)
{
    constexpr size_t kSmem = PipeSmem<K, LR + LT>::kBytes;
    const K cin = (K)xor_in, cout = (K)xor_out;
    if (mode == 2) {
        if (hP)
            k_pipe<1, K, LR, LT><<<grid, 1 << LT, kSmem, s>>>((K*)base, lo, hi, *hP, ntiles, cin, cout, status);
        else
            k_pipe_big<1, K, LR, LT><<<grid, 1 << LT, kSmem, s>>>((K*)base, lo, hi, dP, ntiles, cin, cout, status);
    } else {
        if (hP)
            k_pipe<0, K, LR, LT><<<grid, 1 << LT, kSmem, s>>>((K*)base, lo, hi, *hP, ntiles, cin, cout, status);
        else
            k_pipe_big<0, K, LR, LT><<<grid, 1 << LT, kSmem, s>>>((K*)base, lo, hi, dP, ntiles, cin, cout, status);
    }
    return cudaGetLastError();
}

template <typename K, int LR, int LT>
cudaError_t pipe_attr_t(int* blocks_per_sm)
{
    constexpr int kSmem = (int)PipeSmem<K, LR + LT>::kBytes;
    cudaError_t e = cudaSuccess;
    for (auto fn : {k_pipe<0, K, LR, LT>, k_pipe<1, K, LR, LT>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    for (auto fn : {k_pipe_big<0, K, LR, LT>, k_pipe_big<1, K, LR, LT>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_pipe<0, K, LR, LT>, 1 << LT, kSmem);
    return e;
}

// Configurations compiled in pipelined form (the others report zero CTAs
// per SM and run one CTA per tile).
#define BITONIC_PIPE_CONFIGS(X) \
    X(0, uint32_t, 6, 8, 1)     \
    X(1, uint32_t, 5, 8, 1)     \
    X(4, uint64_t, 5, 8, 1)

}  // namespace

cudaError_t launch_pipe(int mode, int cfg, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                        const TileParamsBig* dP, uint32_t ntiles, uint32_t grid, uint64_t xor_in,
                        uint64_t xor_out, int* status, cudaStream_t s)
{
#define BITONIC_PIPE_CASE(ID, KT, LR, LT, MB)                                                                 \
    case ID:                                                                                                \
        return launch_pipe_t<KT, LR, LT>(mode, base, lo, hi, hP, dP, ntiles, grid, xor_in, xor_out, \
                                         status, s);
    switch (cfg) {
        BITONIC_PIPE_CONFIGS(BITONIC_PIPE_CASE)
        default: return cudaErrorInvalidValue;
    }
#undef BITONIC_PIPE_CASE
}

cudaError_t set_pipe_wait(uint32_t max_spins, int starve)
{
    if (max_spins == 0) max_spins = kMaxWaitSpins;
    cudaError_t e = cudaMemcpyToSymbol(g_pipe_wait_spins, &max_spins, sizeof(max_spins));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_pipe_starve, &starve, sizeof(starve));
    return e;
}

// Sets the shared-memory limit of every pipelined kernel on the current
// device and reports each configuration's resident CTAs per SM (0 = not
// available in pipelined form).
cudaError_t init_pipe_attributes(int* blocks_per_sm)
{
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kNumTileCfgs; ++i) blocks_per_sm[i] = 0;
#define BITONIC_PIPE_ATTR(ID, KT, LR, LT, MB) \
    if (e == cudaSuccess) e = pipe_attr_t<KT, LR, LT>(&blocks_per_sm[ID]);
    BITONIC_PIPE_CONFIGS(BITONIC_PIPE_ATTR)
#undef BITONIC_PIPE_ATTR
    return e;
}

}  // namespace bitonic
