// Tile-kernel configurations compiled into the library: (id, key type,
// log2 keys per thread, log2 threads per CTA).  A tile holds
// 2^(log_r + log_t) keys in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "desc.h"

// (id, key type, log2 keys per thread, log2 threads, resident CTAs per SM
// the registers are capped for: 1 = no cap)
#define BITONIC_TILE_CONFIGS_U32(X)                                          \
    X(0, uint32_t, 6, 8, 1)  /* 16K keys, 256 threads x 64 keys */          \
    X(1, uint32_t, 5, 8, 1)  /*  8K keys, 256 threads x 32 keys */          \
    X(2, uint32_t, 5, 9, 1)  /* 16K keys, 512 threads x 32 keys */          \
    X(3, uint32_t, 3, 10, 1) /*  8K keys, 1024 threads x 8 keys (semi) */   \
    X(7, uint32_t, 6, 8, 3)  /* 16K keys, 256 x 64, capped for 3 CTAs/SM */

#define BITONIC_TILE_CONFIGS_U64(X)                                          \
    X(4, uint64_t, 5, 8, 1)  /*  8K composites, 256 threads x 32 */         \
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

// Tile launches; complement_in / complement_out complement the keys on load /
// store (descending 4-byte sorts run ascending on ~key).
cudaError_t launch_tile(int cfg, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                        const TileParamsBig* dP, uint32_t grid, int complement_in, int complement_out,
                        cudaStream_t s, uint32_t pf_dist = 0);
cudaError_t launch_tile_u32(int cfg, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                            const TileParamsBig* dP, uint32_t grid, int complement_in, int complement_out,
                            uint32_t pf_dist, cudaStream_t s);
cudaError_t launch_tile_u64(int cfg, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                            const TileParamsBig* dP, uint32_t grid, int complement_in, int complement_out,
                            uint32_t pf_dist, cudaStream_t s);
cudaError_t tile_blocks_per_sm_u32(int cfg, int* blocks);
cudaError_t tile_blocks_per_sm_u64(int cfg, int* blocks);
cudaError_t tile_blocks_per_sm(int cfg, int* blocks);
cudaError_t init_tile_attributes_u32();
cudaError_t init_tile_attributes_u64();
cudaError_t launch_pipe(int mode, int cfg, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                        const TileParamsBig* dP, uint32_t ntiles, uint32_t grid, int complement_in,
                        int complement_out, int* status, cudaStream_t s);
cudaError_t init_pipe_attributes(int* blocks_per_sm);
cudaError_t launch_step(int key_bytes, int desc, void* base, uint32_t lo, uint32_t hi, uint32_t N, int j,
                        int flip, cudaStream_t s);

}  // namespace bitonic
