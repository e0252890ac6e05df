// Tile-kernel configurations compiled into the library: (id, key type,
// log2 keys per thread, log2 threads per CTA).  A tile holds
// 2^(log_r + log_t) keys in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "desc.h"

#define BITONIC_TILE_CONFIGS(X)                                         \
    X(0, uint32_t, 6, 8)  /* 16K keys, 256 threads x 64 keys */         \
    X(1, uint32_t, 5, 8)  /*  8K keys, 256 threads x 32 keys */         \
    X(2, uint32_t, 5, 9)  /* 16K keys, 512 threads x 32 keys */         \
    X(3, uint32_t, 3, 10) /*  8K keys, 1024 threads x 8 keys (semi) */  \
    X(4, uint64_t, 5, 8)  /*  8K composites, 256 threads x 32 */        \
    X(5, uint64_t, 4, 8)  /*  4K composites, 256 threads x 16 */        \
    X(6, uint64_t, 2, 10) /*  4K composites, 1024 threads x 4 (semi) */ \
    X(7, uint32_t, 6, 9)  /* 32K keys, 512 threads x 64 keys */         \
    X(8, uint32_t, 5, 10) /* 32K keys, 1024 threads x 32 keys */        \
    X(9, uint64_t, 5, 9)  /* 16K composites, 512 threads x 32 */      \
    X(10, uint32_t, 7, 7) /* 16K keys, 128 threads x 128 keys */       \
    X(11, uint64_t, 6, 7) /*  8K composites, 128 threads x 64 */

namespace bitonic {

struct TileCfg {
    int id;
    int key_bytes;
    int log_r;
    int log_t;
};

constexpr int kNumTileCfgs = 12;

cudaError_t launch_tile(int cfg, int desc, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                        const TileParamsBig* dP, uint32_t grid, cudaStream_t s);
cudaError_t launch_pipe(int cfg, int desc, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                        const TileParamsBig* dP, uint32_t ntiles, uint32_t grid, int* status, cudaStream_t s);
cudaError_t init_pipe_attributes(int* blocks_per_sm);
cudaError_t launch_step(int key_bytes, int desc, void* base, uint32_t lo, uint32_t hi, uint32_t N, int j,
                        int flip, cudaStream_t s);

}  // namespace bitonic
