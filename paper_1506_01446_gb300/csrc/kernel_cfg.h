// Tile-kernel configurations compiled into the library: (id, key type,
// log2 keys per thread, log2 threads per CTA).  A tile holds
// 2^(log_r + log_t) keys in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "desc.h"

// (id, key type, log2 keys per thread, log2 threads, resident CTAs per SM
// the registers are bounded for: 1 = no bound, 2 = two, 3 = three (the
// "capped" kernels, which spill a little))
#define BITONIC_TILE_CONFIGS_U32(X)                                          \
    X(0, uint32_t, 6, 8, 2)  /* 16K keys, 256 threads x 64 keys */          \
    X(1, uint32_t, 5, 8, 1)  /*  8K keys, 256 threads x 32 keys */          \
    X(2, uint32_t, 5, 9, 1)  /* 16K keys, 512 threads x 32 keys */          \
    X(3, uint32_t, 3, 10, 1) /*  8K keys, 1024 threads x 8 keys (semi) */   \
    X(7, uint32_t, 6, 8, 3)  /* 16K keys, 256 x 64, capped for 3 CTAs/SM */

#define BITONIC_TILE_CONFIGS_U64(X)                                          \
    X(4, uint64_t, 5, 8, 2)  /*  8K composites, 256 threads x 32 */         \
    X(5, uint64_t, 4, 8, 1)  /*  4K composites, 256 threads x 16 */         \
    X(6, uint64_t, 2, 10, 1) /*  4K composites, 1024 threads x 4 (semi) */  \
    X(8, uint64_t, 5, 8, 3)  /*  8K composites, capped for 3 CTAs/SM */

#define BITONIC_TILE_CONFIGS(X) BITONIC_TILE_CONFIGS_U32(X) BITONIC_TILE_CONFIGS_U64(X)

namespace bitonic {

struct TileCfg {
    int id;
    int key_bytes;
    int log_r;
    int log_t;
    int min_blocks;
};

constexpr int kNumTileCfgs = 9;

const TileCfg& tile_cfg(int id);

// Host side of an order-preserving key map v -> v ^ (fill(v ^ s) & a) ^ b
// (fill = all ones if the top bit is set), truncated to the key width at
// launch; the device side is KeyMap in engine.cuh.  All zero: identity.
struct KeyMapHost {
    uint64_t a = 0, b = 0, s = 0;
};

// Tile launches; real keys pass through mi on load and mo on store.  CTA i
// of the launch runs tile cta0 + i of the pass (a launch may cover a range).
cudaError_t launch_tile(int cfg, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                        const TileParamsBig* dP, uint32_t grid, const KeyMapHost& mi, const KeyMapHost& mo,
                        cudaStream_t s, uint32_t pf_dist = 0, uint32_t cta0 = 0);
cudaError_t launch_tile_u32(int cfg, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                            const TileParamsBig* dP, uint32_t grid, const KeyMapHost& mi, const KeyMapHost& mo,
                            uint32_t pf_dist, uint32_t cta0, cudaStream_t s);
cudaError_t launch_tile_u64(int cfg, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                            const TileParamsBig* dP, uint32_t grid, const KeyMapHost& mi, const KeyMapHost& mo,
                            uint32_t pf_dist, uint32_t cta0, cudaStream_t s);
// Applies a key map to base[lo, hi) in one elementwise pass (for launch
// kinds that cannot fuse it: the one-step kernels, the pipelined kernels
// with a float map).
cudaError_t launch_keymap(int key_bytes, void* base, uint32_t lo, uint32_t hi, const KeyMapHost& m, cudaStream_t s);
cudaError_t tile_blocks_per_sm_u32(int cfg, int* blocks);
cudaError_t tile_blocks_per_sm_u64(int cfg, int* blocks);
cudaError_t tile_blocks_per_sm(int cfg, int* blocks);
cudaError_t init_tile_attributes_u32();
cudaError_t init_tile_attributes_u64();
// Pipelined tile launches; keys are XORed with xor_in on load and xor_out on
// store (maps with a = 0 only).
cudaError_t launch_pipe(int mode, int cfg, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                        const TileParamsBig* dP, uint32_t ntiles, uint32_t grid, uint64_t xor_in,
                        uint64_t xor_out, int* status, cudaStream_t s);
cudaError_t init_pipe_attributes(int* blocks_per_sm);
// Bound of the pipelined kernels' mbarrier waits on the current device (0 =
// the default), and their copy-starving test mode.
cudaError_t set_pipe_wait(uint32_t max_spins, int starve);
cudaError_t launch_step(int key_bytes, int desc, void* base, uint32_t lo, uint32_t hi, uint32_t N, int j,
                        int flip, cudaStream_t s);

// Pair sorts on 64-bit composites (key' << 32) | index, key' = key ^ flip.
// The first tile launch builds the composites while it loads the caller's
// keys; the last one splits them while it stores: keys to keys_out, original
// indices to idx_out.
struct PairIo {
    const uint32_t* keys_in;
    uint32_t* keys_out;
    uint32_t* idx_out;    // n indices, 16-byte aligned (workspace)
    uint32_t flip;        // 0 ascending, all ones descending
    uint32_t aligned8;    // keys 8-byte aligned: two-element vector accesses
};

// Composite tile configurations that have the fused pair kernels.
bool tile_pairs_supported(int cfg);
// mode bit 0: build composites on load; bit 1: split on store.  The launch
// covers composites [0, hi) (no front padding).
cudaError_t launch_tile_pairs(int cfg, int mode, uint64_t* comp, uint32_t hi, const TileParams* hP, uint32_t grid,
                              const PairIo& pio, uint32_t pf_dist, cudaStream_t s);
cudaError_t init_tile_pairs_attributes();
// out[i] = vals[idx[i]] for i < n (out and idx 16-byte aligned), in
// gather_launches(n) launches: above a size the sources are taken in slices
// that fit L2, one launch per slice.
cudaError_t launch_gather_by_index(uint32_t* out, const uint32_t* vals, const uint32_t* idx, uint32_t n,
                                   cudaStream_t s);
int gather_launches(uint32_t n);

}  // namespace bitonic
