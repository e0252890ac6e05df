// Internal declarations shared by the library's translation units (host side).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bitonic.h"
#include "desc.h"

namespace bitonic {

// Kind of one launch in a sort's launch sequence.
enum LaunchKind : int {
    KIND_TILE_SORT = 0,   // phases 1..t of every tile, on chip (Section 4.1 + 4.2)
    KIND_GLOBAL = 1,      // strides 2^hi..2^lo of one phase, several per HBM pass (Section 4.2)
    KIND_TILE_MERGE = 2,  // strides 2^(t-1)..1 of one phase, on chip (Section 4.1)
    KIND_STEP = 3,        // one step, one compare-exchange per thread (Section 3.3)
};

// One kernel launch of a sort of N = 2^k (virtual) positions.  Steps use the
// "mirror" form of the network: the first step of phase p pairs i with
// i ^ (2^p - 1), later steps pair i with i ^ 2^j, and the lower position
// always receives the element that sorts first.  Global bit j of an index is
// the stride 2^j.
struct Launch {
    int kind;
    int phase;   // p, 1-based (tile sort: last phase done)
    int hi;      // highest stride bit handled (tile sort: its last phase's top bit)
    int lo;      // lowest stride bit handled
    int flip;    // 1 if the launch starts with phase p's mirror step (hi == p - 1)
    int desc;    // index into Plan::descs (-1 for KIND_STEP)
    uint32_t grid;
    bool small;  // descriptor fits in TileParams (passed by value)
};

struct Plan {
    bool ok = false;
    uint64_t N = 0;
    int k = 0;
    int cfg = -1;           // tile kernel configuration (kernel_cfg.h), -1 = step kernels
    int tile_log2 = 0;
    std::vector<Launch> launches;
    std::vector<TileParamsBig> descs;  // one per tile launch
    std::vector<TileParams> small;     // by-value copies (valid where Launch::small)
    int hbm_passes = 0;     // launches that stream every key through HBM once
    int fused_steps = 0;    // network steps done on chip
    int global_steps = 0;   // network steps done by global passes
};

struct Options {
    int variant = 0;
    int tile_log2 = 0;
    int global_bits = 0;
    int use_graph = 1;
    int keys_per_thread_log2 = 0;
    int io_direct = 0;
    int l2_prefetch = 1;
    int min_row_log2 = 0;
    int ctas_per_sm = 0;
    int pipeline = 0;
    int round_sync = 0;   // 0: warp barriers where a transpose keeps each warp's slots; 1: CTA barriers
    int split_log2 = 1;   // graph captures: the leading launches as 2^split_log2 concurrent tile ranges
};

// Builds the launch sequence for a sort of n keys of key_bytes bytes.
Plan make_plan(uint64_t n, int key_bytes, const Options& opt);

const struct TileCfg& tile_cfg(int id);

// Packed segmented tiles: descriptor for segments padded to 2^k positions
// (key_bytes 4: 16K-key or, tile_log2 = 13, 8K-key tile; 8: 8K-composite tile).
bool make_class_desc(int key_bytes, int k, TileParamsBig& P, int tile_log2 = 14);

// Launchers (kernels.cu).  Return the CUDA error of the launch.
cudaError_t launch_pairs_pack(uint64_t* comp, const uint32_t* keys, uint32_t n, int desc,
                              cudaStream_t s);
cudaError_t launch_pairs_gather(uint64_t* comp, const uint32_t* vals, uint32_t n, cudaStream_t s);
cudaError_t launch_pairs_unpack(const uint64_t* comp, uint32_t* keys, uint32_t* vals, uint32_t n,
                                int desc, cudaStream_t s);

cudaError_t init_tile_attributes();

// Graph replay mode of the calling host thread (bitonic_set_thread_graphs).
int thread_graph_mode();

// Sets the calling thread's last error message; returns st.
bitonic_status report_error(bitonic_status st, const std::string& what);

}  // namespace bitonic
