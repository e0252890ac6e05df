// C ABI of the library: argument checks, per-stream workspaces, plan and
// CUDA-graph caches, and the launch sequences of each entry point.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "bitonic.h"
#include "internal.h"
#include "kernel_cfg.h"
#include "seg.h"

namespace bitonic {
namespace {

thread_local std::string t_last_error;
// Graph replay for calls from this host thread: -1 = the process-wide
// use_graph option, 0 = plain launches, 1 = replay cached graphs.
thread_local int t_graph_mode = -1;

// Device status word values.
constexpr int kDevOk = 0;
constexpr int kDevBadOffsets = 1;
constexpr int kDevTimeout = 2;

constexpr size_t kMaxGraphs = 64;
constexpr int kMaxSplit = 4;  // most concurrent tile ranges of a split sort (Options::split_log2 <= 2)
// Bound of each wait of the long-segment sort for a segment's previous pass
// (polls about 128 ns apart: about half a second).
constexpr uint32_t kLongWaitSpins = 1u << 22;
constexpr uint64_t kMaxKeys = uint64_t(1) << 31;
// Host-buffer sorts upload, tile-sort, final-pass and download in this many
// chunks, so that copies overlap the passes that need only their own tiles.
constexpr int kHostChunks = 8;

std::mutex g_mu;  // guards every piece of state below
Options g_opt;

struct StreamWs {
    int* dev = nullptr;          // [0] status word, [1] work counter, [2..4] segment stats
    int* host = nullptr;         // pinned copy of the stats
    uint64_t* comp = nullptr;    // pair composites
    size_t comp_cap = 0;         // in elements
    void* seg = nullptr;         // segmented batch plan, class bytes and class order
    size_t seg_cap = 0;          // in bytes
    // host-buffer sorts: a second stream (uploads and downloads stay on the
    // caller's stream, the tile passes run here) and chunk events
    cudaStream_t side = nullptr;
    cudaEvent_t ev[2 * kHostChunks + 1] = {};
    // batched host-buffer sorts: upload and download streams, a second
    // device buffer, and per-buffer chunk / free events
    cudaStream_t up = nullptr, down = nullptr;
    uint32_t* buf2 = nullptr;
    size_t buf2_cap = 0;  // in keys
    cudaEvent_t bev[2][2 * kHostChunks + 1] = {};
    cudaEvent_t bstart = nullptr;
};

struct PlanEntry {
    Plan plan;
    Options opt;                       // options the plan was built with
    TileParamsBig* d_descs = nullptr;  // device copies, used by launches too big to pass by value
};

// Packed-tile choices of a segmented batch, per (pairs, ceil(log2 nseg))
// class, set by the autotuner: tile size, smallest size class (m - gap) and
// resident CTAs per SM of the persistent grid.  Zero fields: defaults.
struct SegOpt {
    int tile_log2 = 0;  // keys: 14 (16K keys, 256 x 64) or 13 (8K, 256 x 32); pairs: 13
    int floor_gap = 0;  // 1..10 (default 10: up to 1024 segments per tile)
    int ctas_per_sm = 0;  // 1 or 2 (default 2)
};
std::map<std::pair<int, int>, SegOpt> g_seg_opt;

SegOpt resolve_seg_options(bool pairs, int nseg)
{
    int c = 0;
    while ((1ll << c) < (long long)nseg) ++c;
    SegOpt o;
    auto it = g_seg_opt.find({pairs ? 1 : 0, c});
    if (it != g_seg_opt.end()) o = it->second;
    if (!o.tile_log2) o.tile_log2 = pairs ? 13 : 14;
    if (!o.floor_gap) o.floor_gap = 10;
    if (!o.ctas_per_sm) o.ctas_per_sm = 2;
    return o;
}

// Per-size-class overrides set by the autotuner: (key bytes, log2 N) -> options.
std::map<std::pair<int, int>, Options> g_class_opt;

// Options for a sort of N = 2^k keys of key_bytes bytes: the size class's
// tuned choice of tile, keys per thread and strides per pass where one is
// set, the process-wide options otherwise.
Options resolve_options(int key_bytes, int k)
{
    auto it = g_class_opt.find({key_bytes, k});
    if (it == g_class_opt.end() || g_opt.variant != 0) return g_opt;
    Options o = g_opt;
    o.tile_log2 = it->second.tile_log2;
    o.keys_per_thread_log2 = it->second.keys_per_thread_log2;
    o.global_bits = it->second.global_bits;
    o.pipeline = it->second.pipeline;
    o.l2_prefetch = it->second.l2_prefetch;
    o.min_row_log2 = it->second.min_row_log2;
    o.ctas_per_sm = it->second.ctas_per_sm;
    return o;
}

// Packs every option that changes a plan into one key (5 bits per field).
uint64_t options_code(const Options& o)
{
    const int f[] = {o.variant, o.tile_log2, o.keys_per_thread_log2, o.global_bits, o.io_direct,
                     o.pipeline, o.l2_prefetch, o.min_row_log2, o.ctas_per_sm, o.round_sync, o.split_log2};
    uint64_t c = 0;
    for (int v : f) c = (c << 5) | uint64_t(v & 31);
    return c;
}

using PlanKey = std::tuple<uint64_t, int, uint64_t>;  // N, key bytes, options_code
// op, n, ascending, ptr a, ptr b, ptr c, count, stream, options_code, unused
using GraphKey = std::tuple<int, uint64_t, int, uintptr_t, uintptr_t, uintptr_t, int, uintptr_t, int, uint64_t, int>;

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    uint64_t stamp = 0;
};

struct DeviceState {
    bool inited = false;
    cudaStream_t capture = nullptr;
    int num_sms = 0;
    int pipe_blocks[kNumTileCfgs] = {};  // resident pipelined CTAs per SM, per configuration
    int tile_blocks[kNumTileCfgs] = {};  // resident tile CTAs per SM, per configuration
    int* status = nullptr;               // device status word shared by every stream
    // forked launch ranges of graph-captured sorts (Options::split_log2)
    cudaStream_t split[kMaxSplit - 1] = {};
    cudaEvent_t split_ev[kMaxSplit] = {};
    // the same for plain launches: a second stream and fork / join events
    // per caller stream, so that sorts on different streams never share one
    struct DirectSplit {
        cudaStream_t stream = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
    };
    std::map<cudaStream_t, DirectSplit> direct_split;
    // packed segment tiles by class: 16K keys, 8K composites (pairs), 8K keys
    TileParamsBig* seg_descs[3] = {nullptr, nullptr, nullptr};
    // Segments longer than one tile (keys): the launch plans of sorts of
    // 2^k keys, k = 15..31, built at the first segmented call.
    bool long_ready[2] = {false, false};  // keys, pairs
    LongPlans long_plans[2] = {};
    TileParamsBig* long_descs[2] = {nullptr, nullptr};
    std::map<cudaStream_t, StreamWs> ws;
    std::map<PlanKey, std::unique_ptr<PlanEntry>> plans;
    std::map<GraphKey, GraphEntry> graphs;
    uint64_t clock = 0;
};

std::map<int, DeviceState> g_dev;

int debug_checks()
{
    static int v = [] {
        const char* e = std::getenv("BITONIC_DEBUG_CHECKS");
        return (e && e[0] == '1') ? 1 : 0;
    }();
    return v;
}

bitonic_status cuda_fail(cudaError_t e, const char* what)
{
    t_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // clear a sticky launch error
    return e == cudaErrorMemoryAllocation ? BITONIC_ERR_OOM : BITONIC_ERR_CUDA;
}

#define BT_CK(call)                                      \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

bitonic_status device_state(DeviceState** out)
{
    int dev = 0;
    BT_CK(cudaGetDevice(&dev));
    DeviceState& ds = g_dev[dev];
    if (!ds.inited) {
        BT_CK(cudaDeviceGetAttribute(&ds.num_sms, cudaDevAttrMultiProcessorCount, dev));
        BT_CK(init_tile_attributes());
        BT_CK(init_pipe_attributes(ds.pipe_blocks));
        for (int c = 0; c < kNumTileCfgs; ++c) BT_CK(tile_blocks_per_sm(c, &ds.tile_blocks[c]));
        BT_CK(seg_init_attributes());
        BT_CK(cudaStreamCreateWithFlags(&ds.capture, cudaStreamNonBlocking));
        for (cudaStream_t& t : ds.split) BT_CK(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
        for (cudaEvent_t& e : ds.split_ev) BT_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        BT_CK(cudaMalloc(&ds.status, sizeof(int)));
        BT_CK(cudaMemset(ds.status, 0, sizeof(int)));
        for (int which = 0; which < 3; ++which) {
            const int kb = which == 1 ? 8 : 4, m = which == 0 ? 14 : 13;
            std::vector<TileParamsBig> descs(m + 1);
            std::memset(descs.data(), 0, descs.size() * sizeof(TileParamsBig));
            for (int k = 1; k <= m; ++k)
                if (!make_class_desc(kb, k, descs[k], m)) return BITONIC_ERR_UNSUPPORTED;
            BT_CK(cudaMalloc(&ds.seg_descs[which], descs.size() * sizeof(TileParamsBig)));
            BT_CK(cudaMemcpy(ds.seg_descs[which], descs.data(), descs.size() * sizeof(TileParamsBig),
                             cudaMemcpyHostToDevice));
        }
        ds.inited = true;
    }
    *out = &ds;
    return BITONIC_OK;
}

// Descriptors of the plain sorts of 2^k keys, k = m..31 (default options),
// for the long segments of a segmented batch: keys (pairs = 0) on 16K-key
// tiles, m = 14 (k = 14, one tile, only when the packed tiles hold 8K keys);
// pairs on 8K-composite tiles, m = 13, whose schedules add a pack pass
// before the plan and gather and split passes after it.
bitonic_status ensure_long_plans(DeviceState& ds, int pairs)
{
    if (ds.long_ready[pairs]) return BITONIC_OK;
    LongPlans lp = {};
    lp.tile_log = pairs ? 13 : 14;
    const int extra = pairs ? 3 : 0;
    std::vector<TileParamsBig> descs;
    const Options o;
    for (int k = lp.tile_log; k <= 31; ++k) {
        const Plan pl = make_plan(uint64_t(1) << k, pairs ? 8 : 4, o);
        if (!pl.ok || pl.cfg != (pairs ? 4 : 0) || (int)pl.launches.size() + extra > kLongMaxPasses) {
            t_last_error = "long-segment plans";
            return BITONIC_ERR_UNSUPPORTED;
        }
        lp.npass[k] = (int)pl.launches.size() + extra;
        lp.desc0[k] = (int)descs.size();
        for (const Launch& L : pl.launches) {
            if (L.desc < 0 || L.grid != (1u << (k - lp.tile_log))) {
                t_last_error = "long-segment plans";
                return BITONIC_ERR_UNSUPPORTED;
            }
            descs.push_back(pl.descs[L.desc]);
        }
    }
    const size_t bytes = descs.size() * sizeof(TileParamsBig);
    BT_CK(cudaMalloc(&ds.long_descs[pairs], bytes));
    BT_CK(cudaMemcpy(ds.long_descs[pairs], descs.data(), bytes, cudaMemcpyHostToDevice));
    ds.long_plans[pairs] = lp;
    ds.long_ready[pairs] = true;
    return BITONIC_OK;
}

bool stream_capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cst) != cudaSuccess) return false;
    return cst != cudaStreamCaptureStatusNone;
}

// Workspace of stream s, grown to hold comp_need composites.  While s is
// being captured nothing can be allocated: the call then uses the stream's
// existing workspace, or else the device's default (NULL-stream) workspace,
// and fails if neither is large enough.
void drop_stream_graphs(DeviceState& ds, cudaStream_t s)
{
    for (auto it = ds.graphs.begin(); it != ds.graphs.end();) {
        if (std::get<7>(it->first) == (uintptr_t)s) {
            cudaGraphExecDestroy(it->second.exec);
            it = ds.graphs.erase(it);
        } else {
            ++it;
        }
    }
}

bitonic_status stream_ws(DeviceState& ds, cudaStream_t s, size_t comp_need, StreamWs** out, size_t seg_need = 0)
{
    if (stream_capturing(s)) {
        for (cudaStream_t key : {s, (cudaStream_t) nullptr}) {
            auto it = ds.ws.find(key);
            if (it != ds.ws.end() && it->second.dev && it->second.comp_cap >= comp_need &&
                it->second.seg_cap >= seg_need) {
                *out = &it->second;
                return BITONIC_OK;
            }
        }
        t_last_error = "no workspace large enough for a captured call: run the same call once outside capture";
        return BITONIC_ERR_UNSUPPORTED;
    }
    StreamWs& w = ds.ws[s];
    if (!w.dev) {
        BT_CK(cudaMalloc(&w.dev, 8 * sizeof(int)));
        BT_CK(cudaMemset(w.dev, 0, 8 * sizeof(int)));
        BT_CK(cudaMallocHost(&w.host, 8 * sizeof(int)));
    }
    if (comp_need > w.comp_cap) {
        if (w.comp) {
            BT_CK(cudaStreamSynchronize(s));
            BT_CK(cudaFree(w.comp));
            w.comp = nullptr;
            w.comp_cap = 0;
            drop_stream_graphs(ds, s);  // graphs captured with the old buffer must not be replayed
        }
        size_t cap = (comp_need + 1) & ~size_t(1);
        BT_CK(cudaMalloc(&w.comp, cap * sizeof(uint64_t)));
        w.comp_cap = cap;
    }
    if (seg_need > w.seg_cap) {
        if (w.seg) {
            BT_CK(cudaStreamSynchronize(s));
            BT_CK(cudaFree(w.seg));
            w.seg = nullptr;
            w.seg_cap = 0;
            drop_stream_graphs(ds, s);
        }
        BT_CK(cudaMalloc(&w.seg, seg_need));
        w.seg_cap = seg_need;
    }
    *out = &w;
    return BITONIC_OK;
}

bitonic_status get_plan(DeviceState& ds, uint64_t nv, int key_bytes, PlanEntry** out)
{
    uint64_t N = 2;
    int k = 1;
    while (N < nv) { N <<= 1; ++k; }
    const Options o = resolve_options(key_bytes, k);
    PlanKey key{N, key_bytes, options_code(o)};
    auto it = ds.plans.find(key);
    if (it == ds.plans.end()) {
        auto pe = std::make_unique<PlanEntry>();
        pe->opt = o;
        pe->plan = make_plan(N, key_bytes, o);
        if (!pe->plan.ok) {
            t_last_error = "planner could not schedule this size";
            return BITONIC_ERR_UNSUPPORTED;
        }
        bool need_big = false;
        for (const Launch& L : pe->plan.launches) need_big |= (L.desc >= 0 && !L.small);
        if (need_big) {
            const size_t bytes = pe->plan.descs.size() * sizeof(TileParamsBig);
            BT_CK(cudaMalloc(&pe->d_descs, bytes));
            BT_CK(cudaMemcpy(pe->d_descs, pe->plan.descs.data(), bytes, cudaMemcpyHostToDevice));
        }
        it = ds.plans.emplace(key, std::move(pe)).first;
    }
    *out = it->second.get();
    return BITONIC_OK;
}

// Enqueues the plan's launches on `s`.  events / kinds are optional.
// Key types of the keys-only sorts.  The network always sorts ascending on
// unsigned integers; every other type and direction reaches that order by an
// order-preserving map on the first load and its inverse on the last store
// (KeyMapHost; the device side is KeyMap in engine.cuh).
enum KeyType { KEY_U32 = 0, KEY_I32 = 1, KEY_F32 = 2, KEY_U64 = 3, KEY_I64 = 4, KEY_F64 = 5 };

struct KeyMaps {
    KeyMapHost in, out;
};

int key_type_bytes(int type) { return type >= KEY_U64 ? 8 : 4; }

// Maps for a type and direction, on keys of w bits (sign = the top bit):
//   unsigned       v ^ b, b = 0 (ascending) or all ones (descending);
//   signed         v ^ b, b = sign (ascending) or ~sign (descending);
//   IEEE 754 float v ^ (fill(v) & ~sign) ^ sign: negative keys have every bit
//                  flipped, non-negative ones the sign bit, so totalOrder
//                  becomes unsigned order; descending also complements.
//                  The inverse reads the sign from ~v (s = all ones).
KeyMaps key_maps(int type, int ascending)
{
    const int w = 8 * key_type_bytes(type);
    const uint64_t ones = w == 64 ? ~0ull : 0xFFFFFFFFull;
    const uint64_t sign = 1ull << (w - 1);
    KeyMaps m;
    switch (type) {
    case KEY_U32:
    case KEY_U64:
        m.in.b = m.out.b = ascending ? 0 : ones;
        break;
    case KEY_I32:
    case KEY_I64:
        m.in.b = m.out.b = ascending ? sign : (ones & ~sign);
        break;
    default:  // floats
        m.in.a = m.out.a = ones & ~sign;
        m.in.b = ascending ? sign : (ones & ~sign);
        m.out.b = ascending ? sign : 0;
        m.out.s = ones;
        break;
    }
    return m;
}

// Pair sorts build their composites in the first tile launch and split them
// in the last one (PairIo) when the plan runs on tile kernels of a composite
// configuration that has those kernels, with by-value descriptors; otherwise
// separate pack, gather and split kernels surround the plan.
bool pairs_fused(const Plan& pl, const Options& o)
{
    return !pl.launches.empty() && pl.launches[0].kind != KIND_STEP && !o.pipeline && tile_pairs_supported(pl.cfg) &&
           pl.launches.front().small && pl.launches.back().small;
}

// Smallest tile count of a launch that splits: below it the extra
// launches (and, outside a graph, the fork and join) cost more than the
// tails they fill.  2^20 keys in plain launches: 0.151 split against 0.131
// ms; 2^22: 0.223 against 0.197; 2^24: 0.583 against 0.674.  In a graph
// 2^17..2^21 keys are 3-5% slower split, 2^22 the same, 2^23 13% faster.
constexpr uint32_t kSplitMinTilesGraph = 256, kSplitMinTilesPlain = 1024;

// End of the run of launches from launch i that a graph-captured sort
// splits into S concurrent tile ranges (see enqueue_plan); i when the launch
// at i starts no such run (runs are at least two launches long).  pairs_io:
// the plan's first and last launches build and split pair composites and
// stay whole.
size_t split_run_end(const Plan& pl, size_t i, int S, int split_log2, bool pairs_io)
{
    if (S < 2) return i;
    const size_t nl = pl.launches.size();
    size_t e = i;
    while (e < nl) {
        const Launch& L = pl.launches[e];
        const bool edge = pairs_io && (e == 0 || e + 1 == nl);
        if (L.kind == KIND_STEP || edge || L.hi >= pl.k - split_log2 || L.grid % (uint32_t)S != 0) break;
        ++e;
    }
    return e - i >= 2 ? e : i;
}

bitonic_status enqueue_plan(DeviceState& ds, const PlanEntry& pe, void* base, uint32_t lo, uint32_t hi,
                            const KeyMaps& km, int key_bytes, int* status, cudaStream_t s, cudaEvent_t* events,
                            int* kinds, const PairIo* pio = nullptr)
{
    const Plan& pl = pe.plan;
    const uint64_t ones = key_bytes == 8 ? ~0ull : 0xFFFFFFFFull;
    const bool xor_only = km.in.a == 0 && km.out.a == 0;
    const bool steps = !pl.launches.empty() && pl.launches[0].kind == KIND_STEP;
    const bool piped = pe.opt.pipeline && ds.pipe_blocks[pl.cfg] > 0 && status;
    // The one-step kernels run ascending or descending on raw 4-byte keys
    // themselves; the pipelined kernels take XOR masks.  Any other map runs
    // as a separate elementwise pass before the first and after the last
    // launch.
    int step_desc = 0;
    bool separate = false;
    if (steps) {
        const bool plain = xor_only && km.in.b == km.out.b && (km.in.b == 0 || (km.in.b == ones && key_bytes == 4));
        if (plain) step_desc = km.in.b != 0;
        else separate = true;
    } else if (piped && !xor_only) {
        separate = true;
    }
    const KeyMapHost ident;
    if (separate) {
        cudaError_t e = launch_keymap(key_bytes, base, lo, hi, km.in, s);
        if (e != cudaSuccess) return cuda_fail(e, "key map launch");
    }
    const size_t nl = pl.launches.size();
    auto pmode_of = [&](size_t i) { return pio ? ((i == 0 ? 1 : 0) | (i + 1 == nl ? 2 : 0)) : 0; };
    auto live_tiles = [&](const Launch& L) {  // tiles wholly past the last key have nothing to do
        const TileParamsBig& D = pl.descs[L.desc];
        uint32_t ntiles = L.grid;
        if (D.contiguous) {
            const uint64_t live = ((uint64_t)hi + (1u << D.m) - 1) >> D.m;
            if (live < ntiles) ntiles = (uint32_t)live;
        }
        return ntiles;
    };
    const uint32_t wave = (uint32_t)(pe.opt.l2_prefetch * ds.tile_blocks[pl.cfg] * ds.num_sms);
    // Concurrent tile ranges (Options::split_log2); in a graph the forked
    // streams become parallel branches: a launch whose strides all lie below bit k - split_log2
    // works within blocks of 2^(k - split_log2) positions, and since a
    // tile's index fills the position bits outside the tile from the lowest
    // up, part q of the array is tile range [q T / S, (q + 1) T / S).  A run
    // of such launches goes to S streams, each taking its part through the
    // whole run; the streams join back before the next launch.  Two parts
    // (the default): 2^28 keys 12.04 against 12.12 ms, 2^24 0.565 against
    // 0.626 ms (each launch's last wave overlaps the other part's next
    // launch).  Four parts were slower (2^28: 13.02 ms), and so was a second
    // part started one launch behind the first (12.12 ms).
    // The library's own captures split into S parts on its shared fork
    // streams (s is then ds.capture): those captures begin and end inside
    // one call under the library's lock.  Plain launches split in two on a
    // second stream of the caller's stream's own.  Launches that go straight
    // into a caller's capture stay whole: a stream forked into a caller's
    // capture would stay part of it until the caller ends it.
    int S = 1;
    cudaStream_t fork_streams[kMaxSplit - 1] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[kMaxSplit - 1] = {};
    const uint32_t tiles = nl ? pl.launches[0].grid : 0;
    if (pe.opt.split_log2 > 0 && pe.opt.variant == 0 && !steps && !piped && !events &&
        tiles >= kSplitMinTilesGraph) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        BT_CK(cudaStreamIsCapturing(s, &cst));
        if (s == ds.capture && cst == cudaStreamCaptureStatusActive) {
            S = 1 << pe.opt.split_log2;
            for (int q = 0; q + 1 < S; ++q) {
                fork_streams[q] = ds.split[q];
                join_ev[q] = ds.split_ev[q + 1];
            }
            fork_ev = ds.split_ev[0];
        } else if (cst == cudaStreamCaptureStatusNone && tiles >= kSplitMinTilesPlain) {
            DeviceState::DirectSplit& d = ds.direct_split[s];
            if (!d.stream) {
                BT_CK(cudaStreamCreateWithFlags(&d.stream, cudaStreamNonBlocking));
                BT_CK(cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming));
                BT_CK(cudaEventCreateWithFlags(&d.join, cudaEventDisableTiming));
            }
            S = 2;
            fork_streams[0] = d.stream;
            fork_ev = d.fork;
            join_ev[0] = d.join;
        }
    }
    const int split_log2 = S == 4 ? 2 : (S == 2 ? 1 : 0);
    for (size_t i = 0; i < nl;) {
        const size_t run_end = split_run_end(pl, i, S, split_log2, pio != nullptr);
        if (run_end > i) {
            BT_CK(cudaEventRecord(fork_ev, s));
            for (int q = 1; q < S; ++q) BT_CK(cudaStreamWaitEvent(fork_streams[q - 1], fork_ev, 0));
            for (int q = 0; q < S; ++q) {
                cudaStream_t sq = q == 0 ? s : fork_streams[q - 1];
                for (size_t a = i; a < run_end; ++a) {
                    const Launch& L = pl.launches[a];
                    const TileParams* hP = L.small ? &pl.small[L.desc] : nullptr;
                    const TileParamsBig* dP = L.small ? nullptr : pe.d_descs + L.desc;
                    const uint32_t per = L.grid / (uint32_t)S, ntiles = live_tiles(L);
                    const uint32_t t0 = (uint32_t)q * per, t1 = std::min(t0 + per, ntiles);
                    if (t1 <= t0) continue;
                    const KeyMapHost& mi = (a == 0 && !separate) ? km.in : ident;
                    const KeyMapHost& mo = (a + 1 == nl && !separate) ? km.out : ident;
                    cudaError_t e = launch_tile(pl.cfg, base, lo, hi, hP, dP, t1 - t0, mi, mo, sq, wave, t0);
                    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
                }
            }
            for (int q = 1; q < S; ++q) {
                BT_CK(cudaEventRecord(join_ev[q - 1], fork_streams[q - 1]));
                BT_CK(cudaStreamWaitEvent(s, join_ev[q - 1], 0));
            }
            i = run_end;
            continue;
        }
        const Launch& L = pl.launches[i];
        if (events) BT_CK(cudaEventRecord(events[i], s));
        if (kinds) kinds[i] = L.kind;
        cudaError_t e;
        if (L.kind == KIND_STEP) {
            e = launch_step(key_bytes, step_desc, base, lo, hi, (uint32_t)pl.N, L.hi, L.flip, s);
        } else {
            const TileParams* hP = L.small ? &pl.small[L.desc] : nullptr;
            const TileParamsBig* dP = L.small ? nullptr : pe.d_descs + L.desc;
            const uint32_t ntiles = live_tiles(L);
            // The key maps are fused into the first load and the last store.
            const KeyMapHost& mi = (i == 0 && !separate) ? km.in : ident;
            const KeyMapHost& mo = (i + 1 == nl && !separate) ? km.out : ident;
            const int pmode = pmode_of(i);
            if (pmode) {
                e = launch_tile_pairs(pl.cfg, pmode, (uint64_t*)base, hi, hP, ntiles, *pio, wave, s);
            } else if (piped) {
                const int per_sm = ds.pipe_blocks[pl.cfg];
                uint64_t g = (uint64_t)per_sm * ds.num_sms;
                const uint32_t grid = (uint32_t)(g < ntiles ? g : ntiles);
                e = launch_pipe(pe.opt.pipeline, pl.cfg, base, lo, hi, hP, dP, ntiles, grid, mi.b, mo.b, status, s);
            } else {
                e = launch_tile(pl.cfg, base, lo, hi, hP, dP, ntiles, mi, mo, s, wave);
            }
        }
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        ++i;
    }
    if (events) BT_CK(cudaEventRecord(events[pl.launches.size()], s));
    if (separate) {
        cudaError_t e = launch_keymap(key_bytes, base, lo, hi, km.out, s);
        if (e != cudaSuccess) return cuda_fail(e, "key map launch");
    }
    return BITONIC_OK;
}

template <class F>
bitonic_status run_graphed(DeviceState& ds, const GraphKey& key, cudaStream_t user, F&& enqueue)
{
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    BT_CK(cudaStreamIsCapturing(user, &cst));
    const bool graphs = t_graph_mode < 0 ? g_opt.use_graph != 0 : t_graph_mode != 0;
    if (!graphs || cst != cudaStreamCaptureStatusNone) return enqueue(user);
    auto it = ds.graphs.find(key);
    if (it == ds.graphs.end()) {
        BT_CK(cudaStreamBeginCapture(ds.capture, cudaStreamCaptureModeThreadLocal));
        bitonic_status st = enqueue(ds.capture);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(ds.capture, &g);
        if (st != BITONIC_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        if (ds.graphs.size() >= kMaxGraphs) {
            auto victim = ds.graphs.begin();
            for (auto jt = ds.graphs.begin(); jt != ds.graphs.end(); ++jt)
                if (jt->second.stamp < victim->second.stamp) victim = jt;
            BT_CK(cudaDeviceSynchronize());
            cudaGraphExecDestroy(victim->second.exec);
            ds.graphs.erase(victim);
        }
        it = ds.graphs.emplace(key, GraphEntry{ex, 0}).first;
    }
    it->second.stamp = ++ds.clock;
    BT_CK(cudaGraphLaunch(it->second.exec, user));
    return BITONIC_OK;
}

bitonic_status check_keys_ptr(const void* p, int key_bytes = 4)
{
    if (!p || ((uintptr_t)p & (uintptr_t)(key_bytes - 1))) {
        t_last_error = "null or misaligned pointer";
        return BITONIC_ERR_INVALID;
    }
    return BITONIC_OK;
}

// Keys-only sort of any key type, in place on the caller's stream.
bitonic_status sort_keys_impl(void* keys, size_t n, int type, int ascending, cudaStream_t s, cudaEvent_t* events,
                              int nevents, int* kinds)
{
    if (n > kMaxKeys) return BITONIC_ERR_UNSUPPORTED;
    if (n <= 1) return BITONIC_OK;
    const int kb = key_type_bytes(type);
    bitonic_status st = check_keys_ptr(keys, kb);
    if (st) return st;
    // virtual front padding back to the 16-byte boundary before the keys
    const uint32_t front = (uint32_t)(((uintptr_t)keys & 15u) / (uintptr_t)kb);
    const uint64_t nv = (uint64_t)n + front;
    if (nv > kMaxKeys) return BITONIC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> g(g_mu);
    DeviceState* ds;
    if ((st = device_state(&ds))) return st;
    PlanEntry* pe;
    if ((st = get_plan(*ds, nv, kb, &pe))) return st;
    void* base = (char*)keys - (size_t)front * kb;
    const KeyMaps km = key_maps(type, ascending);
    int* status = ds->status;
    if (events) {
        if (nevents < (int)pe->plan.launches.size() + 1) return BITONIC_ERR_INVALID;
        return enqueue_plan(*ds, *pe, base, front, (uint32_t)nv, km, kb, status, s, events, kinds);
    }
    GraphKey key{type == KEY_U32 ? 0 : 20 + type, n, ascending ? 0 : 1, (uintptr_t)keys, 0, 0, 0, 0, 0,
                 options_code(pe->opt), 0};
    return run_graphed(*ds, key, s, [&](cudaStream_t cs) {
        return enqueue_plan(*ds, *pe, base, front, (uint32_t)nv, km, kb, status, cs, nullptr, nullptr);
    });
}

// Tile launch i of a plan restricted to its tiles [t0, t1) (non-pipelined).
cudaError_t launch_plan_tiles(const DeviceState& ds, const PlanEntry& pe, size_t i, void* base, uint32_t lo,
                              uint32_t hi, const KeyMapHost& mi, const KeyMapHost& mo, cudaStream_t s, uint32_t t0,
                              uint32_t t1)
{
    const Plan& pl = pe.plan;
    const Launch& L = pl.launches[i];
    const TileParams* hP = L.small ? &pl.small[L.desc] : nullptr;
    const TileParamsBig* dP = L.small ? nullptr : pe.d_descs + L.desc;
    const uint32_t pf = pe.opt.l2_prefetch > 0
                            ? (uint32_t)(pe.opt.l2_prefetch * ds.tile_blocks[pl.cfg] * ds.num_sms)
                            : 0u;
    return launch_tile(pl.cfg, base, lo, hi, hP, dP, t1 - t0, mi, mo, s, pf, t0);
}

// Host-buffer sort of one array through the device buffer `dev`, for a plan
// whose first launch is a tile sort on contiguous tiles.  The upload runs on
// `up` in n_up chunks and each chunk's tiles are sorted on `comp` once they
// arrive; the other launches follow on `comp`; the download runs on `down`
// in n_down chunks, each as soon as the last launch has finished its tiles
// (when that launch works on contiguous tiles; otherwise after it).  Chunk
// counts are capped at kHostChunks and at the tile count; ev_in / ev_out hold
// kHostChunks events each.  The caller orders the streams after earlier work.
// Phases of enqueue_host_sort: the upload, the passes and the download can
// be enqueued separately (the passes wait on the upload's chunk events, the
// download on the passes' chunk events), so that a batch can put the next
// array's upload ahead of this array's download.
constexpr int kHostUpload = 1, kHostCompute = 2, kHostDownload = 4;

bitonic_status enqueue_host_sort(DeviceState& ds, const PlanEntry& pe, const uint32_t* in, uint32_t* out,
                                 size_t n, const KeyMaps& km, uint32_t* dev, cudaStream_t up, cudaStream_t comp,
                                 cudaStream_t down, cudaEvent_t* ev_in, cudaEvent_t* ev_out, int n_up, int n_down,
                                 int phases = kHostUpload | kHostCompute | kHostDownload)
{
    const Plan& pl = pe.plan;
    const size_t L = pl.launches.size();
    const TileParamsBig& first = pl.descs[pl.launches[0].desc];
    const bool last_tiled = pl.descs[pl.launches[L - 1].desc].contiguous;
    const int m = first.m;
    const uint32_t live = (uint32_t)((n + (size_t(1) << m) - 1) >> m);  // tiles holding real keys
    auto chunks = [&](int want) {
        const uint32_t c = (uint32_t)std::max(1, std::min(want, kHostChunks));
        return live < c ? live : c;
    };
    const uint32_t nin = chunks(n_up), nout = chunks(L == 1 ? n_up : n_down);
    auto tiles_of = [&](uint32_t c, uint32_t nch) { return (uint32_t)((uint64_t)live * c / nch); };
    auto keys_of = [&](uint32_t t) { return std::min<size_t>((size_t)t << m, n); };
    const KeyMapHost ident;
    // With C = nin a power of two dividing the T tiles of every launch,
    // upload chunk c is tiles [c T / C, (c + 1) T / C): part c of the sort's
    // positions.  A launch whose strides all lie below bit k - log2(C) works
    // within those parts (a tile's index fills the position bits outside the
    // tile from the lowest up), so the leading run of such launches runs on
    // each chunk as soon as it has arrived, overlapping the rest of the
    // upload; the other launches follow over all tiles.
    const uint32_t T = pl.launches[0].grid;
    int lc = 0;
    while ((2u << lc) <= nin) ++lc;
    size_t prefix = 0;
    if (nin > 1 && (1u << lc) == nin && T % nin == 0 && L > 1)
        while (prefix + 1 < L && pl.launches[prefix].kind != KIND_STEP && pl.launches[prefix].hi < pl.k - lc)
            ++prefix;
    auto in_tiles = [&](uint32_t c) {
        return prefix ? std::min<uint32_t>((uint32_t)((uint64_t)T * c / nin), live) : tiles_of(c, nin);
    };
    // The same at the end: with D = nout a power of two dividing T, the
    // trailing run of launches whose strides stay below bit k - log2(D)
    // (at least the last launch, a tile merge on contiguous tiles) runs per
    // download chunk, and each chunk is downloaded as soon as its part is
    // done.  L: no such run (the last launch is chunked on its own).
    int lo2 = 0;
    while ((2u << lo2) <= nout) ++lo2;
    size_t suffix = L;
    if (L > 1 && nout > 1 && (1u << lo2) == nout && T % nout == 0 && last_tiled) {
        const size_t first_free = prefix ? prefix : 1;
        suffix = L;
        while (suffix > first_free && pl.launches[suffix - 1].kind != KIND_STEP &&
               pl.launches[suffix - 1].hi < pl.k - lo2)
            --suffix;
    }
    auto out_tiles = [&](uint32_t c) {
        return suffix < L ? std::min<uint32_t>((uint32_t)((uint64_t)T * c / nout), live) : tiles_of(c, nout);
    };
    // upload in chunks; the tile sort (launch 0) follows each chunk
    if (phases & kHostUpload)
        for (uint32_t c = 0; c < nin; ++c) {
            const size_t a = keys_of(in_tiles(c)), b = keys_of(in_tiles(c + 1));
            BT_CK(cudaMemcpyAsync(dev + a, in + a, (b - a) * sizeof(uint32_t), cudaMemcpyHostToDevice, up));
            BT_CK(cudaEventRecord(ev_in[c], up));
        }
    if ((phases & kHostCompute) && nin == 1 && nout == 1 && L > 1) {
        // one upload and one download: the whole plan as the cached graph of
        // the device sort of these keys (with its leading launches split in
        // concurrent halves), replayed on the compute stream
        BT_CK(cudaStreamWaitEvent(comp, ev_in[0], 0));
        const GraphKey key{0, (uint64_t)n, km.in.b != 0 ? 1 : 0, (uintptr_t)dev, 0, 0, 0, 0, 0, options_code(pe.opt), 0};
        bitonic_status st = run_graphed(ds, key, comp, [&](cudaStream_t cs) {
            return enqueue_plan(ds, pe, dev, 0, (uint32_t)n, km, 4, ds.status, cs, nullptr, nullptr);
        });
        if (st != BITONIC_OK) return st;
        BT_CK(cudaEventRecord(ev_out[0], comp));
    } else if (phases & kHostCompute) {
        // tiles of launch i that hold real keys
        auto live_of = [&](size_t i) {
            const TileParamsBig& D = pl.descs[pl.launches[i].desc];
            const uint32_t g = pl.launches[i].grid;
            return D.contiguous ? std::min<uint32_t>(g, (uint32_t)((n + (size_t(1) << D.m) - 1) >> D.m)) : g;
        };
        // launches [i0, i1) on part c of C parts (tiles [c T / C, (c + 1) T / C))
        auto run_part = [&](size_t i0, size_t i1, uint32_t c, uint32_t C) -> bitonic_status {
            const uint32_t t0 = (uint32_t)((uint64_t)T * c / C), t1 = (uint32_t)((uint64_t)T * (c + 1) / C);
            if (t0 >= live) return BITONIC_OK;  // only virtual padding in this part
            for (size_t i = i0; i < i1; ++i) {
                const uint32_t end = std::min(t1, live_of(i));
                if (end <= t0) continue;
                cudaError_t e = launch_plan_tiles(ds, pe, i, dev, 0, (uint32_t)n, i == 0 ? km.in : ident,
                                                  i + 1 == L ? km.out : ident, comp, t0, end);
                if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
            }
            return BITONIC_OK;
        };
        size_t start = 1;
        if (prefix) {  // the leading run on each upload chunk as soon as it has arrived
            for (uint32_t c = 0; c < nin; ++c) {
                BT_CK(cudaStreamWaitEvent(comp, ev_in[c], 0));
                bitonic_status st = run_part(0, prefix, c, nin);
                if (st != BITONIC_OK) return st;
            }
            start = prefix;
        } else {  // the tile sort on each upload chunk
            for (uint32_t c = 0; c < nin; ++c) {
                BT_CK(cudaStreamWaitEvent(comp, ev_in[c], 0));
                const bool also_last = L == 1;
                cudaError_t e = launch_plan_tiles(ds, pe, 0, dev, 0, (uint32_t)n, km.in, also_last ? km.out : ident,
                                                  comp, tiles_of(c, nin), tiles_of(c + 1, nin));
                if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
                if (also_last) BT_CK(cudaEventRecord(ev_out[c], comp));
            }
        }
        if (L > 1) {
            // the middle launches over all tiles, then the trailing run per
            // download chunk (suffix), else the last launch alone
            const size_t tail = suffix < L ? suffix : L - 1;
            for (size_t i = start; i < tail; ++i) {
                cudaError_t e = launch_plan_tiles(ds, pe, i, dev, 0, (uint32_t)n, ident, ident, comp, 0, live_of(i));
                if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
            }
            if (suffix < L) {
                for (uint32_t c = 0; c < nout; ++c) {
                    bitonic_status st = run_part(suffix, L, c, nout);
                    if (st != BITONIC_OK) return st;
                    BT_CK(cudaEventRecord(ev_out[c], comp));
                }
            } else if (last_tiled) {
                for (uint32_t c = 0; c < nout; ++c) {
                    cudaError_t e = launch_plan_tiles(ds, pe, L - 1, dev, 0, (uint32_t)n, ident, km.out, comp,
                                                      tiles_of(c, nout), tiles_of(c + 1, nout));
                    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
                    BT_CK(cudaEventRecord(ev_out[c], comp));
                }
            } else {
                const Launch& Ll = pl.launches[L - 1];
                cudaError_t e = launch_plan_tiles(ds, pe, L - 1, dev, 0, (uint32_t)n, ident, km.out, comp, 0, Ll.grid);
                if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
                for (uint32_t c = 0; c < nout; ++c) BT_CK(cudaEventRecord(ev_out[c], comp));
            }
        }
    }
    if (!(phases & kHostDownload)) return BITONIC_OK;
    // download each chunk once its last launch is done
    for (uint32_t c = 0; c < nout; ++c) {
        const size_t a = keys_of(out_tiles(c)), b = keys_of(out_tiles(c + 1));
        BT_CK(cudaStreamWaitEvent(down, ev_out[c], 0));
        BT_CK(cudaMemcpyAsync(out + a, dev + a, (b - a) * sizeof(uint32_t), cudaMemcpyDeviceToHost, down));
    }
    return BITONIC_OK;
}

// 4-byte keys from host memory: in[0..n) -> out[0..n) (in may equal out).
// The keys go through a per-stream device buffer.  When the plan starts with
// a tile sort on contiguous tiles (every plan of the optimized and semi
// variants), the upload runs in chunks on the caller's stream and each
// chunk's tiles are sorted on a second stream as soon as they arrive; when
// the last launch also works on contiguous tiles, its chunks are downloaded
// as each finishes.  Otherwise upload, sort and download run in turn.
bitonic_status sort_u32_host_impl(const uint32_t* in, uint32_t* out, size_t n, int ascending, cudaStream_t s)
{
    if (n > kMaxKeys) return BITONIC_ERR_UNSUPPORTED;
    if (n == 0) return BITONIC_OK;
    if (!in || !out) {
        t_last_error = "null host pointer";
        return BITONIC_ERR_INVALID;
    }
    std::lock_guard<std::mutex> g(g_mu);
    bitonic_status st;
    if (stream_capturing(s)) {
        t_last_error = "host-buffer sorts are not captured into graphs";
        return BITONIC_ERR_UNSUPPORTED;
    }
    DeviceState* ds;
    if ((st = device_state(&ds))) return st;
    StreamWs* w;
    if ((st = stream_ws(*ds, s, (n + 1) / 2, &w))) return st;
    if (!w->side) {
        BT_CK(cudaStreamCreateWithFlags(&w->side, cudaStreamNonBlocking));
        for (cudaEvent_t& e : w->ev) BT_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    uint32_t* dev = reinterpret_cast<uint32_t*>(w->comp);
    const size_t bytes = n * sizeof(uint32_t);
    if (n == 1) {
        BT_CK(cudaMemcpyAsync(dev, in, bytes, cudaMemcpyHostToDevice, s));
        BT_CK(cudaMemcpyAsync(out, dev, bytes, cudaMemcpyDeviceToHost, s));
        return BITONIC_OK;
    }
    PlanEntry* pe;
    if ((st = get_plan(*ds, n, 4, &pe))) return st;
    const Plan& pl = pe->plan;
    const KeyMaps km = key_maps(KEY_U32, ascending);
    const bool tiles = !pl.launches.empty() && pl.launches[0].kind != KIND_STEP && !pe->opt.pipeline &&
                       pl.descs[pl.launches[0].desc].contiguous;
    if (!tiles) {
        BT_CK(cudaMemcpyAsync(dev, in, bytes, cudaMemcpyHostToDevice, s));
        if ((st = enqueue_plan(*ds, *pe, dev, 0, (uint32_t)n, km, 4, ds->status, s, nullptr, nullptr))) return st;
        BT_CK(cudaMemcpyAsync(out, dev, bytes, cudaMemcpyDeviceToHost, s));
        return BITONIC_OK;
    }
    BT_CK(cudaEventRecord(w->ev[2 * kHostChunks], s));
    BT_CK(cudaStreamWaitEvent(w->side, w->ev[2 * kHostChunks], 0));
    return enqueue_host_sort(*ds, *pe, in, out, n, km, dev, s, w->side, s, w->ev, w->ev + kHostChunks, kHostChunks,
                             kHostChunks);
}

// Batched host-buffer sorts: the arrays alternate between two device
// buffers.  Uploads run on one stream, the passes on a second (one array
// after another), downloads on a third, so that array j+1's upload and
// array j-1's download overlap array j's passes.  A buffer is refilled only
// after its previous download has finished.
bitonic_status sort_u32_host_batch_impl(const uint32_t* const* in, uint32_t* const* out, const size_t* n, int count,
                                        int ascending, cudaStream_t s)
{
    if (count < 0 || (count > 0 && (!in || !out || !n))) {
        t_last_error = "bad batch arrays";
        return BITONIC_ERR_INVALID;
    }
    size_t maxn = 0;
    for (int j = 0; j < count; ++j) {
        if (n[j] > kMaxKeys) return BITONIC_ERR_UNSUPPORTED;
        if (n[j] && (!in[j] || !out[j])) {
            t_last_error = "null host pointer";
            return BITONIC_ERR_INVALID;
        }
        maxn = std::max(maxn, n[j]);
    }
    if (maxn == 0) return BITONIC_OK;
    bitonic_status st;
    {
        std::lock_guard<std::mutex> g(g_mu);
        if (stream_capturing(s)) {
            t_last_error = "host-buffer sorts are not captured into graphs";
            return BITONIC_ERR_UNSUPPORTED;
        }
        DeviceState* ds;
        if ((st = device_state(&ds))) return st;
        StreamWs* w;
        if ((st = stream_ws(*ds, s, (maxn + 1) / 2, &w))) return st;
        if (!w->up) {
            if (!w->side) {
                BT_CK(cudaStreamCreateWithFlags(&w->side, cudaStreamNonBlocking));
                for (cudaEvent_t& e : w->ev) BT_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            }
            BT_CK(cudaStreamCreateWithFlags(&w->up, cudaStreamNonBlocking));
            BT_CK(cudaStreamCreateWithFlags(&w->down, cudaStreamNonBlocking));
            for (auto& row : w->bev)
                for (cudaEvent_t& e : row) BT_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            BT_CK(cudaEventCreateWithFlags(&w->bstart, cudaEventDisableTiming));
        }
        if (maxn > w->buf2_cap) {
            if (w->buf2) {
                BT_CK(cudaStreamSynchronize(s));
                BT_CK(cudaFree(w->buf2));
                w->buf2 = nullptr;
                w->buf2_cap = 0;
            }
            BT_CK(cudaMalloc(&w->buf2, maxn * sizeof(uint32_t)));
            w->buf2_cap = maxn;
        }
        uint32_t* bufs[2] = {reinterpret_cast<uint32_t*>(w->comp), w->buf2};
        const KeyMaps km = key_maps(KEY_U32, ascending);
        BT_CK(cudaEventRecord(w->bstart, s));
        for (cudaStream_t t : {w->up, w->side, w->down}) BT_CK(cudaStreamWaitEvent(t, w->bstart, 0));
        // The arrays that hold keys, in order; they alternate between the two
        // buffers.  Array r+1's upload is enqueued before array r's download,
        // so that it never waits behind that download in a copy queue (the
        // download waits for array r's passes): on one in-order copy engine
        // the other order serialises every step's copies with its passes.
        std::vector<int> real;
        for (int j = 0; j < count; ++j)
            if (n[j]) real.push_back(j);
        const int R = (int)real.size();
        std::vector<PlanEntry*> pes(R, nullptr);
        std::vector<char> tiled(R, 0);
        for (int r = 0; r < R; ++r) {
            const int j = real[r];
            if (n[j] > 1 && (st = get_plan(*ds, n[j], 4, &pes[r]))) return st;
            PlanEntry* pe = pes[r];
            tiled[r] = pe && pe->plan.launches[0].kind != KIND_STEP && !pe->opt.pipeline &&
                       pe->plan.descs[pe->plan.launches[0].desc].contiguous;
        }
        // Once the pipeline is full an array's upload ends long before its
        // passes start and its download overlaps the next array's passes:
        // only the first upload and the last download are chunked (a chunked
        // launch leaves a partial wave per chunk).
        auto phase = [&](int r, int what) -> bitonic_status {
            const int j = real[r], b = r & 1;
            uint32_t* dev = bufs[b];
            cudaEvent_t* ev_in = w->bev[b];
            cudaEvent_t* ev_out = w->bev[b] + kHostChunks;
            cudaEvent_t ev_free = w->bev[b][2 * kHostChunks];
            const size_t bytes = n[j] * sizeof(uint32_t);
            if (what == kHostUpload && r >= 2)
                BT_CK(cudaStreamWaitEvent(w->up, ev_free, 0));  // buffer b's last download is done
            if (tiled[r]) {
                const int n_up = r == 0 ? kHostChunks : 1, n_down = r + 1 == R ? kHostChunks : 1;
                bitonic_status q = enqueue_host_sort(*ds, *pes[r], in[j], out[j], n[j], km, dev, w->up, w->side,
                                                     w->down, ev_in, ev_out, n_up, n_down, what);
                if (q) return q;
            } else if (what == kHostUpload) {
                BT_CK(cudaMemcpyAsync(dev, in[j], bytes, cudaMemcpyHostToDevice, w->up));
                BT_CK(cudaEventRecord(ev_in[0], w->up));
            } else if (what == kHostCompute) {
                BT_CK(cudaStreamWaitEvent(w->side, ev_in[0], 0));
                if (pes[r]) {
                    bitonic_status q = enqueue_plan(*ds, *pes[r], dev, 0, (uint32_t)n[j], km, 4, ds->status,
                                                    w->side, nullptr, nullptr);
                    if (q) return q;
                }
                BT_CK(cudaEventRecord(ev_out[0], w->side));
            } else {
                BT_CK(cudaStreamWaitEvent(w->down, ev_out[0], 0));
                BT_CK(cudaMemcpyAsync(out[j], dev, bytes, cudaMemcpyDeviceToHost, w->down));
            }
            if (what == kHostDownload) BT_CK(cudaEventRecord(ev_free, w->down));
            return BITONIC_OK;
        };
        if (R > 0 && (st = phase(0, kHostUpload))) return st;
        for (int r = 0; r < R; ++r) {
            if ((st = phase(r, kHostCompute))) return st;
            if (r + 1 < R && (st = phase(r + 1, kHostUpload))) return st;
            if ((st = phase(r, kHostDownload))) return st;
        }
        // the caller's stream continues once every download (hence every pass) is done
        BT_CK(cudaEventRecord(w->bstart, w->down));
        BT_CK(cudaStreamWaitEvent(s, w->bstart, 0));
    }
    return BITONIC_OK;
}

bitonic_status sort_pairs_impl(uint32_t* keys, uint32_t* vals, size_t n, int ascending, cudaStream_t s)
{
    if (n > kMaxKeys) return BITONIC_ERR_UNSUPPORTED;
    if (n <= 1) return BITONIC_OK;
    bitonic_status st = check_keys_ptr(keys);
    if (st || (st = check_keys_ptr(vals))) return st;
    std::lock_guard<std::mutex> g(g_mu);
    DeviceState* ds;
    if ((st = device_state(&ds))) return st;
    PlanEntry* pe;
    if ((st = get_plan(*ds, n, 8, &pe))) return st;
    const bool fused = pairs_fused(pe->plan, pe->opt);
    // composites (n, rounded to 16 bytes), then, for the fused kernels, a
    // copy of the values that the last launch gathers from
    const size_t comp_elems = (n + 1) & ~size_t(1);
    StreamWs* w;
    if ((st = stream_ws(*ds, s, fused ? comp_elems + ((n + 3) / 4) * 2 : n, &w))) return st;
    const int desc = ascending ? 0 : 1;
    const uint32_t nn = (uint32_t)n;
    uint64_t* comp = w->comp;
    GraphKey key{1, n, desc, (uintptr_t)keys, (uintptr_t)vals, (uintptr_t)comp, 0, (uintptr_t)s, 0,
                 options_code(pe->opt), 0};
    if (fused) {
        // The last tile launch leaves the original indices after the
        // composites; the values are gathered by index into the composite
        // array (dead by then) and copied back over the caller's values.
        uint32_t* idx = reinterpret_cast<uint32_t*>(comp + comp_elems);
        uint32_t* vtmp = reinterpret_cast<uint32_t*>(comp);
        PairIo pio;
        pio.keys_in = keys;
        pio.keys_out = keys;
        pio.idx_out = idx;
        pio.flip = desc ? 0xFFFFFFFFu : 0u;
        pio.aligned8 = ((uintptr_t)keys & 7u) == 0 ? 1u : 0u;
        return run_graphed(*ds, key, s, [&](cudaStream_t cs) -> bitonic_status {
            bitonic_status st2 = enqueue_plan(*ds, *pe, comp, 0, nn, KeyMaps{}, 8, ds->status, cs, nullptr, nullptr,
                                              &pio);
            if (st2) return st2;
            BT_CK(launch_gather_by_index(vtmp, vals, idx, nn, cs));
            BT_CK(cudaMemcpyAsync(vals, vtmp, (size_t)nn * sizeof(uint32_t), cudaMemcpyDeviceToDevice, cs));
            return BITONIC_OK;
        });
    }
    return run_graphed(*ds, key, s, [&](cudaStream_t cs) -> bitonic_status {
        BT_CK(launch_pairs_pack(comp, keys, nn, desc, cs));
        bitonic_status st2 = enqueue_plan(*ds, *pe, comp, 0, nn, KeyMaps{}, 8, ds->status, cs, nullptr, nullptr);
        if (st2) return st2;
        BT_CK(launch_pairs_gather(comp, vals, nn, cs));
        BT_CK(launch_pairs_unpack(comp, keys, vals, nn, desc, cs));
        return BITONIC_OK;
    });
}

bitonic_status sort_segmented_impl(uint32_t* keys, uint32_t* vals, const int32_t* offsets, int nseg,
                                   cudaStream_t s, int64_t max_len = -1)
{
    if (nseg < 0 || !offsets) {
        t_last_error = "negative segment count or null offsets";
        return BITONIC_ERR_INVALID;
    }
    if (nseg == 0) return BITONIC_OK;
    bitonic_status st = check_keys_ptr(keys);
    if (st) return st;
    if (vals && (st = check_keys_ptr(vals))) return st;
    if ((uintptr_t)offsets & 3u) return BITONIC_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_mu);
    DeviceState* ds;
    if ((st = device_state(&ds))) return st;
    StreamWs* w;
    const size_t seg_need = seg_long_ws_bytes(nseg);
    if ((st = stream_ws(*ds, s, 0, &w, seg_need))) return st;
    if ((st = ensure_long_plans(*ds, vals ? 1 : 0))) return st;
    const SegOpt so = resolve_seg_options(vals != nullptr, nseg);
    const TileParamsBig* class_descs = vals ? ds->seg_descs[1] : ds->seg_descs[so.tile_log2 == 13 ? 2 : 0];
    const uint64_t so_code = (uint64_t)so.tile_log2 << 16 | (uint64_t)so.floor_gap << 8 | (uint64_t)so.ctas_per_sm;
    // persistent packed-tile CTAs: the chosen number resident per SM
    const int tile_grid = so.ctas_per_sm * ds->num_sms;
    if (!vals) {
        GraphKey key{2, 0, 1, (uintptr_t)keys, 0, (uintptr_t)offsets, nseg, (uintptr_t)s, 0, so_code, 0};
        void* ws = w->seg;
        return run_graphed(*ds, key, s, [&](cudaStream_t cs) -> bitonic_status {
            BT_CK(seg_tiles_launch(keys, nullptr, offsets, nseg, ws, class_descs, so.tile_log2, so.floor_gap,
                                   tile_grid, ds->status, debug_checks(), cs));
            // segments longer than one tile: their own multi-pass plans, one persistent launch
            BT_CK(seg_long_launch(LongIo{keys, nullptr, nullptr, 0}, offsets, nseg, ws, ds->long_plans[0],
                                  ds->long_descs[0],
                                  kSegTileBlocksKeys * ds->num_sms, ds->status, kLongWaitSpins, cs));
            return BITONIC_OK;
        });
    }
    // Pairs: segments longer than one tile need a composite workspace sized
    // by the span of the offsets, which is read back first -- unless the
    // caller bounds every segment by one tile.
    if (max_len >= 0 && max_len <= (1 << 13)) {
        void* ws = w->seg;
        BT_CK(seg_tiles_launch(keys, vals, offsets, nseg, ws, class_descs, 13, so.floor_gap, tile_grid,
                               ds->status, debug_checks(), s));
        return BITONIC_OK;
    }
    if (stream_capturing(s)) {
        t_last_error = "segmented pair sort reads its segment sizes back and cannot be captured";
        return BITONIC_ERR_UNSUPPORTED;
    }
    BT_CK(seg_launch_stats(offsets, nseg, w->dev + 2, s));
    BT_CK(cudaMemcpyAsync(w->host, w->dev + 2, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
    BT_CK(cudaStreamSynchronize(s));
    const int32_t first = w->host[0], last = w->host[1], longest = w->host[2];
    size_t need = 0;
    if (longest > (1 << 13) && last > first) need = (size_t)(last - first);
    if ((st = stream_ws(*ds, s, need, &w, seg_need))) return st;
    BT_CK(seg_tiles_launch(keys, vals, offsets, nseg, w->seg, class_descs, 13, so.floor_gap, tile_grid,
                           ds->status, debug_checks(), s));
    // segments longer than one tile: composites in the workspace at their
    // offset from offsets[0], their own multi-pass plans, one persistent launch
    if (longest > (1 << 13))
        BT_CK(seg_long_launch(LongIo{keys, vals, w->comp, first}, offsets, nseg, w->seg, ds->long_plans[1],
                              ds->long_descs[1], kSegTileBlocksPairs * ds->num_sms, ds->status, kLongWaitSpins, s));
    return BITONIC_OK;
}

// Segmented sort in either direction.  Descending: complement the keys of
// the segments' span, sort ascending, complement back (three launches on the
// caller's stream).  Every argument is checked before a key changes.
bitonic_status sort_segmented_dir_impl(uint32_t* keys, uint32_t* vals, const int32_t* offsets, int nseg,
                                       int ascending, cudaStream_t s)
{
    if (ascending) return sort_segmented_impl(keys, vals, offsets, nseg, s);
    if (nseg < 0 || !offsets) {
        t_last_error = "negative segment count or null offsets";
        return BITONIC_ERR_INVALID;
    }
    if (nseg == 0) return BITONIC_OK;
    bitonic_status st = check_keys_ptr(keys);
    if (st) return st;
    if (vals && (st = check_keys_ptr(vals))) return st;
    if ((uintptr_t)offsets & 3u) return BITONIC_ERR_INVALID;
    if (vals && stream_capturing(s)) {
        t_last_error = "segmented pair sort reads its segment sizes back and cannot be captured";
        return BITONIC_ERR_UNSUPPORTED;
    }
    int grid;
    {
        std::lock_guard<std::mutex> g(g_mu);
        DeviceState* ds;
        if ((st = device_state(&ds))) return st;
        grid = 4 * ds->num_sms;
    }
    BT_CK(seg_launch_complement(keys, offsets, nseg, grid, s));
    st = sort_segmented_impl(keys, vals, offsets, nseg, s);
    // complement back also after a failed sort, so that a sort that launched
    // nothing leaves the keys as they were
    const cudaError_t e = seg_launch_complement(keys, offsets, nseg, grid, s);
    if (st) return st;
    BT_CK(e);
    return BITONIC_OK;
}

}  // namespace

int thread_graph_mode() { return t_graph_mode; }

bitonic_status report_error(bitonic_status st, const std::string& what)
{
    t_last_error = what;
    return st;
}

}  // namespace bitonic

using namespace bitonic;

extern "C" {

bitonic_status bitonic_sort_u32(uint32_t* keys, size_t n, int ascending, bitonic_stream_t stream)
{
    return sort_keys_impl(keys, n, KEY_U32, ascending, (cudaStream_t)stream, nullptr, 0, nullptr);
}

bitonic_status bitonic_sort_u32_host(const uint32_t* in, uint32_t* out, size_t n, int ascending,
                                     bitonic_stream_t stream)
{
    return sort_u32_host_impl(in, out, n, ascending, (cudaStream_t)stream);
}

bitonic_status bitonic_sort_u32_host_batch(const uint32_t* const* in, uint32_t* const* out, const size_t* n,
                                           int count, int ascending, bitonic_stream_t stream)
{
    return sort_u32_host_batch_impl(in, out, n, count, ascending, (cudaStream_t)stream);
}

bitonic_status bitonic_sort_i32(int32_t* keys, size_t n, int ascending, bitonic_stream_t stream)
{
    return sort_keys_impl(keys, n, KEY_I32, ascending, (cudaStream_t)stream, nullptr, 0, nullptr);
}

bitonic_status bitonic_sort_f32(float* keys, size_t n, int ascending, bitonic_stream_t stream)
{
    return sort_keys_impl(keys, n, KEY_F32, ascending, (cudaStream_t)stream, nullptr, 0, nullptr);
}

bitonic_status bitonic_sort_u64(uint64_t* keys, size_t n, int ascending, bitonic_stream_t stream)
{
    return sort_keys_impl(keys, n, KEY_U64, ascending, (cudaStream_t)stream, nullptr, 0, nullptr);
}

bitonic_status bitonic_sort_i64(int64_t* keys, size_t n, int ascending, bitonic_stream_t stream)
{
    return sort_keys_impl(keys, n, KEY_I64, ascending, (cudaStream_t)stream, nullptr, 0, nullptr);
}

bitonic_status bitonic_sort_f64(double* keys, size_t n, int ascending, bitonic_stream_t stream)
{
    return sort_keys_impl(keys, n, KEY_F64, ascending, (cudaStream_t)stream, nullptr, 0, nullptr);
}

bitonic_status bitonic_sort_pairs_u32(uint32_t* keys, uint32_t* vals, size_t n, int ascending,
                                      bitonic_stream_t stream)
{
    return sort_pairs_impl(keys, vals, n, ascending, (cudaStream_t)stream);
}

bitonic_status bitonic_sort_segmented_u32(uint32_t* keys, const int32_t* offsets, int nseg,
                                          bitonic_stream_t stream)
{
    return sort_segmented_impl(keys, nullptr, offsets, nseg, (cudaStream_t)stream);
}

bitonic_status bitonic_sort_segmented_pairs_u32(uint32_t* keys, uint32_t* vals, const int32_t* offsets,
                                                int nseg, bitonic_stream_t stream)
{
    if (!vals && nseg > 0) return BITONIC_ERR_INVALID;
    return sort_segmented_impl(keys, vals, offsets, nseg, (cudaStream_t)stream);
}

bitonic_status bitonic_sort_segmented_u32_dir(uint32_t* keys, const int32_t* offsets, int nseg, int ascending,
                                              bitonic_stream_t stream)
{
    return sort_segmented_dir_impl(keys, nullptr, offsets, nseg, ascending, (cudaStream_t)stream);
}

bitonic_status bitonic_sort_segmented_pairs_u32_dir(uint32_t* keys, uint32_t* vals, const int32_t* offsets,
                                                    int nseg, int ascending, bitonic_stream_t stream)
{
    if (!vals && nseg > 0) return BITONIC_ERR_INVALID;
    return sort_segmented_dir_impl(keys, vals, offsets, nseg, ascending, (cudaStream_t)stream);
}

bitonic_status bitonic_sort_segmented_pairs_u32_bounded(uint32_t* keys, uint32_t* vals, const int32_t* offsets,
                                                        int nseg, int max_len, bitonic_stream_t stream)
{
    if (!vals && nseg > 0) return BITONIC_ERR_INVALID;
    if (max_len < 0) return BITONIC_ERR_INVALID;
    return sort_segmented_impl(keys, vals, offsets, nseg, (cudaStream_t)stream, max_len);
}

const char* bitonic_status_string(bitonic_status s)
{
    switch (s) {
        case BITONIC_OK: return "BITONIC_OK";
        case BITONIC_ERR_INVALID: return "BITONIC_ERR_INVALID";
        case BITONIC_ERR_CUDA: return "BITONIC_ERR_CUDA";
        case BITONIC_ERR_OOM: return "BITONIC_ERR_OOM";
        case BITONIC_ERR_TIMEOUT: return "BITONIC_ERR_TIMEOUT";
        case BITONIC_ERR_UNSUPPORTED: return "BITONIC_ERR_UNSUPPORTED";
    }
    return "BITONIC_UNKNOWN_STATUS";
}

const char* bitonic_last_error_message(void) { return t_last_error.c_str(); }

bitonic_status bitonic_last_device_error(bitonic_stream_t stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    BT_CK(cudaStreamSynchronize(s));
    std::lock_guard<std::mutex> g(g_mu);
    int dev = 0;
    BT_CK(cudaGetDevice(&dev));
    auto dit = g_dev.find(dev);
    if (dit == g_dev.end() || !dit->second.status) return BITONIC_OK;
    int word = 0;
    BT_CK(cudaMemcpy(&word, dit->second.status, sizeof(int), cudaMemcpyDeviceToHost));
    BT_CK(cudaMemset(dit->second.status, 0, sizeof(int)));
    if (word == kDevOk) return BITONIC_OK;
    if (word == kDevBadOffsets) return BITONIC_ERR_INVALID;
    if (word == kDevTimeout) return BITONIC_ERR_TIMEOUT;
    return BITONIC_ERR_CUDA;
}

bitonic_status bitonic_release_workspace(void)
{
    std::lock_guard<std::mutex> g(g_mu);
    int dev = 0;
    BT_CK(cudaGetDevice(&dev));
    auto dit = g_dev.find(dev);
    if (dit == g_dev.end()) return BITONIC_OK;
    DeviceState& ds = dit->second;
    BT_CK(cudaDeviceSynchronize());
    for (auto& kv : ds.graphs) cudaGraphExecDestroy(kv.second.exec);
    ds.graphs.clear();
    for (auto& kv : ds.plans)
        if (kv.second->d_descs) cudaFree(kv.second->d_descs);
    ds.plans.clear();
    for (auto& kv : ds.ws) {
        if (kv.second.dev) cudaFree(kv.second.dev);
        if (kv.second.host) cudaFreeHost(kv.second.host);
        if (kv.second.comp) cudaFree(kv.second.comp);
        if (kv.second.seg) cudaFree(kv.second.seg);
        for (cudaEvent_t e : kv.second.ev)
            if (e) cudaEventDestroy(e);
        if (kv.second.side) cudaStreamDestroy(kv.second.side);
        for (auto& row : kv.second.bev)
            for (cudaEvent_t e : row)
                if (e) cudaEventDestroy(e);
        if (kv.second.bstart) cudaEventDestroy(kv.second.bstart);
        if (kv.second.up) cudaStreamDestroy(kv.second.up);
        if (kv.second.down) cudaStreamDestroy(kv.second.down);
        if (kv.second.buf2) cudaFree(kv.second.buf2);
    }
    ds.ws.clear();
    for (auto& kv : ds.direct_split) {
        if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
        if (kv.second.fork) cudaEventDestroy(kv.second.fork);
        if (kv.second.join) cudaEventDestroy(kv.second.join);
    }
    ds.direct_split.clear();
    return BITONIC_OK;
}

bitonic_status bitonic_set_options(const bitonic_options* opt)
{
    if (!opt) return BITONIC_ERR_INVALID;
    if (opt->variant < 0 || opt->variant > 2) return BITONIC_ERR_INVALID;
    if (opt->tile_log2 != 0 && (opt->tile_log2 < 12 || opt->tile_log2 > 15)) return BITONIC_ERR_INVALID;
    if (opt->keys_per_thread_log2 != 0 && (opt->keys_per_thread_log2 < 2 || opt->keys_per_thread_log2 > 7))
        return BITONIC_ERR_INVALID;
    if (opt->global_bits < 0 || opt->global_bits > 16) return BITONIC_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_mu);
    g_opt.variant = opt->variant;
    g_opt.tile_log2 = opt->tile_log2;
    g_opt.global_bits = opt->global_bits;
    g_opt.use_graph = opt->use_graph ? 1 : 0;
    g_opt.keys_per_thread_log2 = opt->keys_per_thread_log2;
    g_opt.pipeline = (opt->pipeline >= 0 && opt->pipeline <= 2) ? opt->pipeline : 0;
    g_opt.io_direct = opt->io_direct & 3;
    g_opt.l2_prefetch = opt->l2_prefetch < 0 ? 0 : (opt->l2_prefetch > 8 ? 8 : opt->l2_prefetch);
    g_opt.min_row_log2 = (opt->min_row_log2 < 0 || opt->min_row_log2 > 12) ? 0 : opt->min_row_log2;
    g_opt.ctas_per_sm = (opt->ctas_per_sm == 2 || opt->ctas_per_sm == 3) ? opt->ctas_per_sm : 0;
    g_opt.round_sync = opt->round_sync ? 1 : 0;
    g_opt.split_log2 = (opt->split_log2 >= 0 && opt->split_log2 <= 2) ? opt->split_log2 : 0;
    return BITONIC_OK;
}

bitonic_status bitonic_debug_set_wait(int starve_copies, unsigned max_spins)
{
    if (starve_copies && max_spins == 0) return BITONIC_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_mu);
    DeviceState* ds;
    bitonic_status st = device_state(&ds);
    if (st) return st;
    BT_CK(cudaDeviceSynchronize());
    // a short bound only together with the starving mode: then no copy is in
    // flight when a wait gives up
    BT_CK(set_pipe_wait(starve_copies ? max_spins : 0u, starve_copies ? 1 : 0));
    return BITONIC_OK;
}

bitonic_status bitonic_set_segmented_options(int pairs, int log2_nseg, const bitonic_seg_options* opt)
{
    if (log2_nseg < 0 || log2_nseg > 31) return BITONIC_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_mu);
    const std::pair<int, int> key{pairs ? 1 : 0, log2_nseg};
    if (!opt) {
        g_seg_opt.erase(key);
        return BITONIC_OK;
    }
    const bool tile_ok = opt->tile_log2 == 0 || opt->tile_log2 == 13 || (!pairs && opt->tile_log2 == 14);
    if (!tile_ok || opt->class_floor_gap < 0 || opt->class_floor_gap > 10 || opt->ctas_per_sm < 0 ||
        opt->ctas_per_sm > 2)
        return BITONIC_ERR_INVALID;
    SegOpt o;
    o.tile_log2 = opt->tile_log2;
    o.floor_gap = opt->class_floor_gap;
    o.ctas_per_sm = opt->ctas_per_sm;
    g_seg_opt[key] = o;
    return BITONIC_OK;
}

bitonic_status bitonic_set_thread_graphs(int mode)
{
    if (mode < -1 || mode > 1) return BITONIC_ERR_INVALID;
    t_graph_mode = mode;
    return BITONIC_OK;
}

bitonic_status bitonic_set_class_options(int key_bytes, int log2_n, const bitonic_options* opt)
{
    if ((key_bytes != 4 && key_bytes != 8) || log2_n < 1 || log2_n > 31) return BITONIC_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_mu);
    if (!opt) {
        g_class_opt.erase({key_bytes, log2_n});
        return BITONIC_OK;
    }
    if (opt->tile_log2 != 0 && (opt->tile_log2 < 12 || opt->tile_log2 > 15)) return BITONIC_ERR_INVALID;
    if (opt->keys_per_thread_log2 != 0 && (opt->keys_per_thread_log2 < 2 || opt->keys_per_thread_log2 > 7))
        return BITONIC_ERR_INVALID;
    if (opt->global_bits < 0 || opt->global_bits > 16 || opt->pipeline < 0 || opt->pipeline > 2)
        return BITONIC_ERR_INVALID;
    Options o;
    o.tile_log2 = opt->tile_log2;
    o.keys_per_thread_log2 = opt->keys_per_thread_log2;
    o.global_bits = opt->global_bits;
    o.pipeline = opt->pipeline;
    o.l2_prefetch = opt->l2_prefetch < 0 ? 0 : (opt->l2_prefetch > 8 ? 8 : opt->l2_prefetch);
    o.min_row_log2 = (opt->min_row_log2 < 0 || opt->min_row_log2 > 12) ? 0 : opt->min_row_log2;
    o.ctas_per_sm = (opt->ctas_per_sm == 2 || opt->ctas_per_sm == 3) ? opt->ctas_per_sm : 0;
    // the planner must accept the choice for this class
    Options probe = g_opt;
    probe.variant = 0;
    probe.tile_log2 = o.tile_log2;
    probe.keys_per_thread_log2 = o.keys_per_thread_log2;
    probe.global_bits = o.global_bits;
    probe.min_row_log2 = o.min_row_log2;
    probe.ctas_per_sm = o.ctas_per_sm;
    if (!make_plan(uint64_t(1) << log2_n, key_bytes, probe).ok) return BITONIC_ERR_UNSUPPORTED;
    g_class_opt[{key_bytes, log2_n}] = o;
    return BITONIC_OK;
}

bitonic_status bitonic_get_options(bitonic_options* opt)
{
    if (!opt) return BITONIC_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_mu);
    opt->variant = g_opt.variant;
    opt->tile_log2 = g_opt.tile_log2;
    opt->global_bits = g_opt.global_bits;
    opt->use_graph = g_opt.use_graph;
    opt->keys_per_thread_log2 = g_opt.keys_per_thread_log2;
    opt->pipeline = g_opt.pipeline;
    opt->io_direct = g_opt.io_direct;
    opt->l2_prefetch = g_opt.l2_prefetch;
    opt->min_row_log2 = g_opt.min_row_log2;
    opt->ctas_per_sm = g_opt.ctas_per_sm;
    opt->round_sync = g_opt.round_sync;
    opt->split_log2 = g_opt.split_log2;
    return BITONIC_OK;
}

bitonic_status bitonic_plan_info(size_t n, int pairs, int* launches, int* hbm_passes, int* fused_steps,
                                 int* global_steps)
{
    if (n > kMaxKeys) return BITONIC_ERR_UNSUPPORTED;
    Options o;
    {
        std::lock_guard<std::mutex> g(g_mu);
        uint64_t N = 2;
        int k = 1;
        while (N < n) { N <<= 1; ++k; }
        o = resolve_options(pairs ? 8 : 4, k);
    }
    if (n <= 1) {
        if (launches) *launches = 0;
        if (hbm_passes) *hbm_passes = 0;
        if (fused_steps) *fused_steps = 0;
        if (global_steps) *global_steps = 0;
        return BITONIC_OK;
    }
    Plan p = make_plan(n, pairs ? 8 : 4, o);
    if (!p.ok) return BITONIC_ERR_UNSUPPORTED;
    if (launches) *launches = (int)p.launches.size() + (pairs ? (pairs_fused(p, o) ? gather_launches((uint32_t)n) : 3) : 0);
    if (hbm_passes) *hbm_passes = p.hbm_passes;
    if (fused_steps) *fused_steps = p.fused_steps;
    if (global_steps) *global_steps = p.global_steps;
    return BITONIC_OK;
}

bitonic_status bitonic_graph_kernels(size_t n, int pairs, int* kernels)
{
    if (!kernels) return BITONIC_ERR_INVALID;
    if (n > kMaxKeys) return BITONIC_ERR_UNSUPPORTED;
    *kernels = 0;
    if (n <= 1) return BITONIC_OK;
    Options o;
    {
        std::lock_guard<std::mutex> g(g_mu);
        uint64_t N = 2;
        int k = 1;
        while (N < n) { N <<= 1; ++k; }
        o = resolve_options(pairs ? 8 : 4, k);
    }
    Plan p = make_plan(n, pairs ? 8 : 4, o);
    if (!p.ok) return BITONIC_ERR_UNSUPPORTED;
    const bool steps = p.launches[0].kind == KIND_STEP;
    const bool fused = pairs && pairs_fused(p, o);
    const int S = (o.split_log2 > 0 && o.variant == 0 && !steps && !o.pipeline &&
                   p.launches[0].grid >= kSplitMinTilesGraph) ? 1 << o.split_log2 : 1;
    int count = 0;
    for (size_t i = 0; i < p.launches.size();) {
        const size_t e = split_run_end(p, i, S, o.split_log2, fused);
        if (e > i) {
            count += (int)(e - i) * S;
            i = e;
        } else {
            ++count;
            ++i;
        }
    }
    if (pairs) count += fused ? gather_launches((uint32_t)n) : 3;
    *kernels = count;
    return BITONIC_OK;
}

bitonic_status bitonic_sort_u32_profiled(uint32_t* keys, size_t n, int ascending, bitonic_stream_t stream,
                                         bitonic_event_t* events, int nevents, int* kinds)
{
    if (!events) return BITONIC_ERR_INVALID;
    return sort_keys_impl(keys, n, KEY_U32, ascending, (cudaStream_t)stream, (cudaEvent_t*)events, nevents, kinds);
}

// Copies the plan of an n-key sort (key_bytes 4 or 8) for inspection:
// info[0] = N, info[1] = cfg id, info[2] = log_r, info[3] = log_t,
// info[4] = launches, info[5] = descriptors; then 7 ints per launch
// (kind, phase, hi, lo, flip, desc, grid).  descs receives up to max_descs
// TileParams.  Host-only: launches nothing.
bitonic_status bitonic_debug_plan(size_t n, int key_bytes, int* info, int max_info, void* descs,
                                  int max_descs)
{
    if (!info || max_info < 6 || (key_bytes != 4 && key_bytes != 8)) return BITONIC_ERR_INVALID;
    if (n > kMaxKeys) return BITONIC_ERR_UNSUPPORTED;
    Options o;
    {
        // the options the sort itself resolves for this size class
        std::lock_guard<std::mutex> g(g_mu);
        uint64_t N = 2;
        int k = 1;
        while (N < n) { N <<= 1; ++k; }
        o = resolve_options(key_bytes, k);
    }
    Plan p = make_plan(n < 2 ? 2 : n, key_bytes, o);
    if (!p.ok) return BITONIC_ERR_UNSUPPORTED;
    info[0] = (int)p.N;
    info[1] = p.cfg;
    info[2] = p.cfg >= 0 ? tile_cfg(p.cfg).log_r : 0;
    info[3] = p.cfg >= 0 ? tile_cfg(p.cfg).log_t : 0;
    info[4] = (int)p.launches.size();
    info[5] = (int)p.descs.size();
    if (max_info < 6 + 7 * (int)p.launches.size() || max_descs < (int)p.descs.size()) return BITONIC_ERR_INVALID;
    for (size_t i = 0; i < p.launches.size(); ++i) {
        const Launch& L = p.launches[i];
        int* o = info + 6 + 7 * i;
        o[0] = L.kind; o[1] = L.phase; o[2] = L.hi; o[3] = L.lo; o[4] = L.flip; o[5] = L.desc; o[6] = (int)L.grid;
    }
    if (descs && !p.descs.empty()) std::memcpy(descs, p.descs.data(), p.descs.size() * sizeof(TileParamsBig));
    return BITONIC_OK;
}

size_t bitonic_debug_desc_size(void) { return sizeof(TileParamsBig); }

}  // extern "C"
