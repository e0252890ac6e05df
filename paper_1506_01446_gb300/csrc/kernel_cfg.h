// Tile-kernel configurations compiled into the library: (id, key type,
// log2 keys per thread, log2 threads per CTA).  A tile holds
// 2^(log_r + log_t) keys in shared memory.
#pragma once

#define BITONIC_TILE_CONFIGS(X)                                         \
    X(0, uint32_t, 6, 8)  /* 16K keys, 256 threads x 64 keys */         \
    X(1, uint32_t, 5, 8)  /*  8K keys, 256 threads x 32 keys */         \
    X(2, uint32_t, 5, 9)  /* 16K keys, 512 threads x 32 keys */         \
    X(3, uint32_t, 3, 10) /*  8K keys, 1024 threads x 8 keys (semi) */  \
    X(4, uint64_t, 5, 8)  /*  8K composites, 256 threads x 32 */        \
    X(5, uint64_t, 4, 8)  /*  4K composites, 256 threads x 16 */        \
    X(6, uint64_t, 2, 10) /*  4K composites, 1024 threads x 4 (semi) */

namespace bitonic {

struct TileCfg {
    int id;
    int key_bytes;
    int log_r;
    int log_t;
};

constexpr int kNumTileCfgs = 7;

cudaError_t launch_tile(int cfg, int desc, void* base, uint32_t lo, uint32_t hi, const struct TileParams* dP,
                        uint32_t grid, cudaStream_t s);
cudaError_t launch_step(int key_bytes, int desc, void* base, uint32_t lo, uint32_t hi, uint32_t N, int j,
                        int flip, cudaStream_t s);

}  // namespace bitonic
