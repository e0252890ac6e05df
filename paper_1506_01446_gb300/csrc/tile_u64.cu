// Tile-pass kernels for 8-byte pair composites.
#include "kernel_cfg.h"
#include "tile_pass.cuh"

namespace bitonic {

cudaError_t launch_tile_u64(int cfg, void* base, uint32_t lo, uint32_t hi, const TileParams* hP,
                            const TileParamsBig* dP, uint32_t grid, const KeyMapHost& mi, const KeyMapHost& mo,
                            uint32_t pf_dist, uint32_t cta0, cudaStream_t s)
{
#define BITONIC_CASE(ID, KT, LR, LT, MB) \
    case ID: return launch_tile_t<KT, LR, LT, MB>(base, lo, hi, hP, dP, grid, mi, mo, pf_dist, cta0, s);
    switch (cfg) {
        BITONIC_TILE_CONFIGS_U64(BITONIC_CASE)
        default: return cudaErrorInvalidValue;
    }
#undef BITONIC_CASE
}

cudaError_t init_tile_attributes_u64()
{
    cudaError_t e = cudaSuccess;
#define BITONIC_ATTR(ID, KT, LR, LT, MB) \
    if (e == cudaSuccess) e = tile_attr_t<KT, LR, LT, MB>();
    BITONIC_TILE_CONFIGS_U64(BITONIC_ATTR)
#undef BITONIC_ATTR
    return e;
}

cudaError_t tile_blocks_per_sm_u64(int cfg, int* blocks)
{
#define BITONIC_OCC(ID, KT, LR, LT, MB) \
    case ID: return tile_occupancy_t<KT, LR, LT, MB>(blocks);
    switch (cfg) {
        BITONIC_TILE_CONFIGS_U64(BITONIC_OCC)
        default: return cudaErrorInvalidValue;
    }
#undef BITONIC_OCC
}

}  // namespace bitonic
