// Segmented-sort launchers (segmented.cu, segmented_tiles.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "desc.h"

namespace bitonic {

constexpr int kSegClasses = 32;       // size classes: k = ceil(log2 length)
constexpr int kSegClassSkip = 30;     // length 0 or 1: nothing to do
constexpr int kSegClassLarge = 31;    // longer than one tile
constexpr int kSegMaxPerTile = 1024;  // segments packed into one tile at most
// Resident CTAs per SM of the packed-tile kernels (registers bounded for it;
// the persistent grid is this many CTAs per SM): 4-byte keys, composites.
// Three for 4-byte keys (80 registers, a few spills) measured 0.78 ms against
// 0.77 ms with two for 65,536 arrays of up to 8192 keys.
constexpr int kSegTileBlocksKeys = 2;
constexpr int kSegTileBlocksPairs = 2;

// Device-side plan of one segmented batch (built by the classify / scan kernels).
struct SegPlan {
    int hist[kSegClasses];            // segments per class
    int seg_start[kSegClasses];       // first position of each class in `order`
    int tile_start[kSegClasses + 1];  // first packed tile of each class
    int cursor[kSegClasses];
    int total_tiles;
    int tile_counter;                 // persistent CTAs' work counter
    int large_counter;
    int pad_;
};

// Segments longer than one packed tile: each runs the full launch plan of a
// sort of N = 2^k keys (its tile sort, multi-stride and merge passes),
// k = ceil(log2(front + length)) >= tile_log, front = the segment's offset
// from a 16-byte boundary.  plans holds, per k, the number of passes of the
// segment's schedule (for pairs the plan's launches plus pack, gather and
// split) and the index of the plan's first descriptor in the device
// descriptor array.
constexpr int kLongMaxPasses = 48;
struct LongPlans {
    int npass[kSegClasses + 1];
    int desc0[kSegClasses + 1];
    int tile_log;  // m: log2 keys per tile of the plans (14 keys, 13 composites)
};

// Arrays of a long-segment launch.  Keys: the tiles run on keys.  Pairs
// (vals != NULL): on 64-bit composites, that of position p (an index into
// keys) at comp[p - comp_first].
struct LongIo {
    uint32_t* keys;
    uint32_t* vals;
    uint64_t* comp;
    int32_t comp_first;
};

// Device-side schedule of one batch's long segments (built per call).
struct LongSched {
    int count[kSegClasses + 1];        // long segments per k
    int class_start[kSegClasses + 1];  // first slot of class k (classes by k descending)
    int cursor[kSegClasses + 1];
    int pass_start[kLongMaxPasses + 1];  // first work item of each pass
    int total_items;
    int work;                          // persistent CTAs' work counter
    int pad_[2];
};

// Workspace of the long-segment sort after the packed-tile one (16-byte aligned).
size_t seg_long_ws_offset(int nseg);
size_t seg_long_ws_bytes(int nseg);
cudaError_t seg_long_init_attributes();
// Sorts the batch's long segments (the packed-tile launch's large class,
// listed in ws) with one persistent launch; max_spins bounds each wait for a
// segment's previous pass.
cudaError_t seg_long_launch(const LongIo& io, const int32_t* offs, int nseg, void* ws, const LongPlans& plans,
                            const TileParamsBig* descs, int grid, int* status, uint32_t max_spins,
                            cudaStream_t s);

cudaError_t seg_init_attributes();
cudaError_t seg_tiles_init_attributes();
size_t seg_tiles_ws_bytes(int nseg);
cudaError_t seg_tiles_launch(uint32_t* keys, uint32_t* vals, const int32_t* offs, int nseg, void* ws,
                             const TileParamsBig* class_descs, int m, int gap, int grid, int* status,
                             int debug_checks, cudaStream_t s);
// out[0] = offsets[0], out[1] = offsets[nseg], out[2] = longest segment.
cudaError_t seg_launch_stats(const int32_t* offs, int nseg, int* out, cudaStream_t s);
// keys[i] = ~keys[i] for i in [offsets[0], offsets[nseg]) (grid-stride).
cudaError_t seg_launch_complement(uint32_t* keys, const int32_t* offs, int nseg, int grid, cudaStream_t s);

}  // namespace bitonic
