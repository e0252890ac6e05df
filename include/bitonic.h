/*
 * bitonic.h -- C ABI of the GB300 (sm_103a) bitonic sorting library.
 *
 * The library sorts 32-bit unsigned keys, key/value pairs, and keys of other
 * types (int32, float, uint64, int64, double), with Batcher's
 * bitonic sorting network as described in "The implementation and
 * optimization of Bitonic sort algorithm based on CUDA" (Mu, Cui, Song;
 * arXiv 1506.01446):
 *   Section 3.1  the network: for n = 2^k, k phases; phase r merges 2^(k-r)
 *                subsequences of length 2^r, each merge taking r half-cleaner
 *                steps of n/2 compare-exchanges;
 *   Section 3.2  k(k+1)/2 steps and n k (k+1) / 4 compare-exchanges in all;
 *   Section 3.3  one kernel per step;
 *   Section 4.1  steps whose subsequences fit in one block's shared memory
 *                are fused into one kernel;
 *   Section 4.2  a thread keeps several elements in registers and applies
 *                successive steps to them without touching global memory.
 *
 * Conventions shared by every entry point
 *   - Pointers named keys / vals / offsets are DEVICE pointers owned by the
 *     caller; they must be aligned to their element size (4 bytes, 8 for
 *     64-bit keys).  Sorting is in place.
 *   - Work is enqueued on `stream` (NULL = the legacy default stream) and the
 *     call returns without waiting.  Argument errors are reported before
 *     anything is enqueued; CUDA launch errors as BITONIC_ERR_CUDA.
 *   - Device-side failures (a bounded wait that ran out, or bad offsets under
 *     BITONIC_DEBUG_CHECKS=1) are written to the device's status word and
 *     reported by bitonic_last_device_error().
 *   - n <= 1 (or nseg == 0) returns BITONIC_OK without launching anything.
 *   - n > 2^31 returns BITONIC_ERR_UNSUPPORTED (indices are 32-bit).
 *   - Sizes that are not powers of two are padded virtually to
 *     N = next_pow2(n): positions >= n behave as keys that sort after every
 *     real key (0xFFFFFFFF ascending); they are never read or written.
 *   - The library owns a per-(device, stream) workspace (pair composites,
 *     work counters; the device buffers, streams and events of the
 *     host-buffer sorts) that grows on demand with cudaMalloc and is freed by
 *     bitonic_release_workspace().  Keys-only device sorts need none.  Calls on
 *     different streams may run concurrently from different host threads;
 *     calls on one stream are serialised by the caller.  While a stream is
 *     being captured nothing is allocated: a pair or segmented call then needs
 *     a workspace from an earlier uncaptured call (on that stream or on the
 *     NULL stream) and returns BITONIC_ERR_UNSUPPORTED otherwise.
 *   - When `stream` is being captured into a CUDA graph, kernels are launched
 *     straight into the capture; otherwise the library replays a cached CUDA
 *     graph of the launch sequence (keyed by size, direction, kind and
 *     buffers).
 */
#ifndef BITONIC_H
#define BITONIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *bitonic_stream_t;
/* Same type as cudaEvent_t. */
typedef struct CUevent_st *bitonic_event_t;

typedef enum {
    BITONIC_OK = 0,
    BITONIC_ERR_INVALID = 1,     /* null pointer, bad flag, negative count, bad alignment */
    BITONIC_ERR_CUDA = 2,        /* a CUDA runtime call failed; see bitonic_last_error_message */
    BITONIC_ERR_OOM = 3,         /* workspace could not be allocated */
    BITONIC_ERR_TIMEOUT = 4,     /* a device-side bounded wait gave up */
    BITONIC_ERR_UNSUPPORTED = 5  /* size beyond the supported range */
} bitonic_status;

/*
 * Sorts keys[0..n) in place, ascending (ascending != 0) or descending.
 * Section 3.1 network (bitonic build + bitonic merge, Section 3.2 work).
 * The output is the unique sorted permutation of the input.
 */
bitonic_status bitonic_sort_u32(uint32_t *keys, size_t n, int ascending, bitonic_stream_t stream);

/*
 * Keys-only sorts of other key types: the same network on the type's own
 * order.  The paper sorts 32-bit integers (Section 5) and names other data
 * types as future work (Section 6); these extend it.
 *   int32 / int64   two's-complement numeric order;
 *   float / double  IEEE 754-2008 totalOrder (clause 5.10):
 *                   -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN, NaNs of
 *                   one sign ordered by payload; bit patterns are preserved;
 *   uint64          unsigned numeric order.
 * Arguments as for bitonic_sort_u32: device pointer, sorted in place, work
 * enqueued on `stream`.  keys must be aligned to the key size
 * (BITONIC_ERR_INVALID otherwise); n up to 2^31 keys (BITONIC_ERR_UNSUPPORTED
 * beyond).  The map to unsigned order is fused into the first load and the
 * last store of the launch sequence (a separate pass only for the basic
 * variant and for floats under the pipelined option).
 */
bitonic_status bitonic_sort_i32(int32_t *keys, size_t n, int ascending, bitonic_stream_t stream);
bitonic_status bitonic_sort_f32(float *keys, size_t n, int ascending, bitonic_stream_t stream);
bitonic_status bitonic_sort_u64(uint64_t *keys, size_t n, int ascending, bitonic_stream_t stream);
bitonic_status bitonic_sort_i64(int64_t *keys, size_t n, int ascending, bitonic_stream_t stream);
bitonic_status bitonic_sort_f64(double *keys, size_t n, int ascending, bitonic_stream_t stream);

/*
 * bitonic_sort_u32 on HOST memory: sorts in[0..n) into out[0..n) (in may
 * equal out).  The paper's timings include the transfers to and from the GPU
 * (Section 5); this call owns them.
 *   - Both pointers are host pointers (page-locked memory gives asynchronous
 *     copies; pageable memory works but the copies then block the caller).
 *   - Work is enqueued on `stream`; out is valid once the stream reaches
 *     that point (synchronise before reading it).
 *   - The keys pass through a per-stream device buffer of 4·n bytes (the
 *     pair workspace, grown with cudaMalloc as needed).
 *   - The upload runs in chunks on `stream`, and each chunk's tiles are
 *     sorted on a library-owned second stream as soon as they arrive.  When
 *     the last pass works on whole tiles, each chunk is downloaded as soon as
 *     its tiles finish.  So the copies overlap the first and last passes.
 *     (Sorts on different streams may run concurrently; for a stream of
 *     arrays bitonic_sort_u32_host_batch overlaps copies with passes
 *     without running two sorts at once.)
 *   - BITONIC_ERR_INVALID for a null pointer when n > 0;
 *     BITONIC_ERR_UNSUPPORTED while `stream` is being captured into a graph,
 *     or for n > 2^31.
 */
bitonic_status bitonic_sort_u32_host(const uint32_t *in, uint32_t *out, size_t n, int ascending,
                                     bitonic_stream_t stream);

/*
 * bitonic_sort_u32_host for count arrays in turn: in[j][0..n[j]) is sorted
 * into out[j][0..n[j]) (host pointers; in[j] may equal out[j]; n[j] = 0
 * skips array j).  The arrays alternate between two device buffers (the
 * second one grown with cudaMalloc to the largest n[j]).  Uploads, passes and
 * downloads run on three library-owned streams: array j+1's upload and
 * array j-1's download overlap array j's passes, while the passes of two
 * arrays never run at once.  `stream` waits for everything before the
 * return; synchronise it before reading out[].  in, out and n are host
 * arrays of count entries.  BITONIC_ERR_INVALID for count < 0 or a null
 * array or pointer; BITONIC_ERR_UNSUPPORTED under graph capture or for
 * n[j] > 2^31.
 */
bitonic_status bitonic_sort_u32_host_batch(const uint32_t *const *in, uint32_t *const *out, const size_t *n,
                                           int count, int ascending, bitonic_stream_t stream);

/*
 * Sorts key/value pairs in place.  Keys compare first; equal keys keep their
 * original index order (ascending index in both directions), so the result is
 * unique.  vals[i] travels with keys[i].  The network is Section 3.1's, run
 * on 64-bit composites (key' << 32) | index, key' = key or ~key, held in a
 * per-stream workspace of about 12 * n bytes: the first tile launch builds
 * the composites while it loads the keys, the last writes the keys back and
 * the original indices to the workspace, a gather kernel reads each value by
 * its index into the workspace and a device copy puts the values back.  (The
 * basic and semi variants use separate pack, gather and split kernels.)
 */
bitonic_status bitonic_sort_pairs_u32(uint32_t *keys, uint32_t *vals, size_t n, int ascending,
                                      bitonic_stream_t stream);

/*
 * Sorts each segment keys[offsets[s] .. offsets[s+1]) ascending, for
 * s = 0..nseg-1, in one batched launch sequence.  `offsets` is a device array
 * of nseg + 1 non-decreasing int32 values (offsets[0] need not be 0); empty
 * segments are allowed.  Offsets are device-resident and are not validated
 * unless the environment variable BITONIC_DEBUG_CHECKS=1 is set, in which
 * case a violation is reported as BITONIC_ERR_INVALID by
 * bitonic_last_device_error().  The segments are binned by size on the
 * device and nothing is read back to the host, so the call is one
 * asynchronous launch sequence (it can be captured in a CUDA graph once a
 * call of the same batch size has sized the stream's workspace).  Segments
 * of up to 16384 keys are packed into shared-memory tiles, many per tile;
 * each longer segment runs the launch plan of a sort of 2^k keys
 * (k = ceil(log2 of its length plus its offset from a 16-byte boundary)):
 * tile sort, multi-stride passes and tile merges.  All of a batch's long
 * segments share one persistent launch whose CTAs take (pass, segment, tile)
 * items in pass order; a tile waits, bounded, until its segment's previous
 * pass is done, and a wait that gives up is reported as BITONIC_ERR_TIMEOUT
 * by bitonic_last_device_error().  A segment longer than 2^31 - 3 keys is
 * reported as BITONIC_ERR_INVALID and left unsorted.
 */
bitonic_status bitonic_sort_segmented_u32(uint32_t *keys, const int32_t *offsets, int nseg,
                                          bitonic_stream_t stream);

/* Segmented key/value sort: each segment sorted ascending by (key, index)
 * with its values, as bitonic_sort_pairs_u32 does for one array.  Segments
 * of up to 8192 pairs are packed into tiles of 64-bit composites; each
 * longer segment runs the launch plan of a 2^k composite sort in a shared
 * persistent launch (as the keys-only call does), with a pack pass before it
 * and gather and split passes after it, its composites in a workspace sized
 * by the span of the offsets.  To size that workspace the call reads three
 * ints back (the offsets' span and the longest segment, one stream
 * synchronisation), so it cannot be captured;
 * bitonic_sort_segmented_pairs_u32_bounded avoids the read-back. */
bitonic_status bitonic_sort_segmented_pairs_u32(uint32_t *keys, uint32_t *vals,
                                                const int32_t *offsets, int nseg,
                                                bitonic_stream_t stream);

/*
 * Segmented sorts in either direction: ascending != 0 is the same call as
 * bitonic_sort_segmented_u32 / bitonic_sort_segmented_pairs_u32; ascending == 0
 * sorts every segment descending (pairs: by key descending, equal keys in
 * ascending original index, as bitonic_sort_pairs_u32 orders them).  A
 * descending sort complements the keys of [offsets[0], offsets[nseg]) on the
 * caller's stream, sorts ascending and complements them back: keys outside
 * that span are not touched (Section 3.1: the network sorts either way).
 * Argument errors, and a pair sort on a capturing stream, are reported
 * before any key changes.  After a later failure the second complement still
 * runs, so a sort that launched nothing leaves the keys as they were.
 */
bitonic_status bitonic_sort_segmented_u32_dir(uint32_t *keys, const int32_t *offsets, int nseg,
                                              int ascending, bitonic_stream_t stream);
bitonic_status bitonic_sort_segmented_pairs_u32_dir(uint32_t *keys, uint32_t *vals,
                                                    const int32_t *offsets, int nseg, int ascending,
                                                    bitonic_stream_t stream);

/*
 * bitonic_sort_segmented_pairs_u32 for callers that know every segment is at
 * most max_len pairs long.  With max_len <= 8192 (one packed tile of 64-bit
 * composites) no segment needs the composite workspace, so nothing is read
 * back to the host and the call is fully asynchronous; larger bounds behave
 * like bitonic_sort_segmented_pairs_u32.  A segment longer than max_len is
 * a caller error (its result is undefined).  Used by the serving loop.
 */
bitonic_status bitonic_sort_segmented_pairs_u32_bounded(uint32_t *keys, uint32_t *vals,
                                                        const int32_t *offsets, int nseg, int max_len,
                                                        bitonic_stream_t stream);

/* Human-readable name of a status code (static storage). */
const char *bitonic_status_string(bitonic_status s);

/* Text of the last CUDA error seen by this host thread ("" if none). */
const char *bitonic_last_error_message(void);

/*
 * Synchronises `stream`, then reads and clears the current device's status
 * word (one per device, shared by every stream), and returns BITONIC_OK,
 * BITONIC_ERR_TIMEOUT or BITONIC_ERR_INVALID (debug offset checks).  Work on
 * other streams that has not finished may still set the word later.
 */
bitonic_status bitonic_last_device_error(bitonic_stream_t stream);

/* Frees every workspace and cached CUDA graph of the current device. */
bitonic_status bitonic_release_workspace(void);

/* ---- planning, tuning and instrumentation (no paper counterpart) -------- */

/* Kernel variants, matching the three GPU columns of Section 5, Table 1. */
typedef enum {
    BITONIC_VARIANT_OPTIMIZED = 0, /* registers + shared memory + multi-stride global passes */
    BITONIC_VARIANT_BASIC = 1,     /* Section 3.3: one kernel per step, one compare-exchange
                                      per thread */
    BITONIC_VARIANT_SEMI = 2       /* Section 4.1: shared-memory tile fusion, one stride per
                                      global pass */
} bitonic_variant;

typedef struct {
    int variant;          /* bitonic_variant */
    int tile_log2;        /* log2 of keys per on-chip tile; 0 = automatic */
    int global_bits;      /* most strides at or above the tile size fused per global pass;
                             0 = automatic (8) */
    int use_graph;        /* 1 = replay cached CUDA graphs (default), 0 = plain launches */
    int keys_per_thread_log2; /* log2 of keys each thread holds in registers; 0 = automatic */
    int io_direct;        /* bit 0: load a tile straight into its first round's register layout,
                             bit 1: store straight from its last round's layout (instead of an
                             extra shared-memory transpose into a coalesced layout); 0 = off */
    int ctas_per_sm;      /* tile kernels: 3 = registers capped for three resident CTAs per SM
                             where such a kernel exists for the tile shape, else two;
                             2 = registers bounded for two CTAs where such a kernel exists,
                             else not bounded; 0 = automatic (2; default) */
    int min_row_log2;     /* shortest run of consecutive keys a multi-stride pass moves, log2
                             (keys); 0 = 128 bytes.  Shorter rows fit one more stride per pass. */
    int l2_prefetch;      /* > 0: each tile CTA asks the TMA unit to prefetch into L2 the tile
                             that many resident waves ahead (default 1); 0 = off */
    int pipeline;         /* 0 = one CTA per tile (default); persistent CTAs that prefetch the
                             next tile into shared memory with 1 = TMA bulk copies per row,
                             2 = per-thread 16-byte cp.async copies */
    int round_sync;       /* tile kernels: 0 = a shared-memory transpose after which every warp
                             reads back exactly the slots it wrote waits at a warp barrier, the
                             others at a CTA barrier (default); 1 = a CTA barrier after every
                             transpose */
    int split_log2;       /* sorts replayed from the library's cached graphs, and plain launches
                             (at most two parts; not the launches that go straight into a
                             caller's own capture): the leading tile launches whose strides stay
                             below 2^(k - split_log2) (every launch before the last split_log2
                             phases) run as 2^split_log2 concurrent tile ranges, one contiguous
                             part of the array each, on library streams that fork from and
                             join back to the sort's stream; 0 = off, 1 (default) or 2 */
} bitonic_options;

/* Process-wide options (defaults: all zero except use_graph = 1, l2_prefetch = 1 and split_log2 = 1). */
bitonic_status bitonic_set_options(const bitonic_options *opt);
bitonic_status bitonic_get_options(bitonic_options *opt);

/*
 * Tuned choice for the packed-tile launch of segmented sorts whose segment
 * count has ceil(log2 nseg) == log2_nseg (pairs != 0: the pair sorts).
 * Written by the autotuner (paper_1506_01446_gb300.autotune); opt == NULL
 * removes the class's choice.  Zero fields keep the defaults.
 */
typedef struct {
    int tile_log2;        /* keys: 14 = 16K-key tiles (256 threads x 64 keys, default) or
                             13 = 8K-key tiles (256 x 32); pairs: 13 (8K composites) */
    int class_floor_gap;  /* 1..10: a segment of L keys is padded to 2^max(ceil(log2 L),
                             tile_log2 - gap) positions, so a tile holds at most 2^gap segments
                             (default 10) */
    int ctas_per_sm;      /* 1 or 2 persistent CTAs per SM (default 2) */
} bitonic_seg_options;

bitonic_status bitonic_set_segmented_options(int pairs, int log2_nseg, const bitonic_seg_options *opt);

/*
 * Graph replay for the calls this host thread makes from now on: mode 1 =
 * replay cached CUDA graphs, 0 = plain launches, -1 = follow the
 * process-wide use_graph option (the default).  Other threads are not
 * affected.  A caller whose buffers change on every call (a server with
 * fresh buffers per request) turns graphs off for its own thread instead of
 * for the whole process.  BITONIC_ERR_INVALID for any other mode.
 */
bitonic_status bitonic_set_thread_graphs(int mode);

/*
 * Testing aid for the device-side failure path (no paper counterpart).
 * starve_copies != 0: from now on every CTA of the pipelined tile kernels
 * (option pipeline = 1) arms its mbarrier for its first tile's bulk copies
 * but issues none of them, and each mbarrier wait gives up after max_spins
 * tries (max_spins >= 1); the kernel then writes BITONIC_ERR_TIMEOUT to the
 * device status word and returns with no copy in flight, so
 * bitonic_last_device_error() reports the timeout and the context stays
 * usable.  starve_copies == 0 restores normal copies and the default bound
 * (max_spins ignored).  Synchronises the device first; the setting applies to
 * the current device.  BITONIC_ERR_INVALID if starve_copies != 0 and
 * max_spins == 0.
 */
bitonic_status bitonic_debug_set_wait(int starve_copies, unsigned max_spins);

/*
 * Tuned choice for one size class: sorts of N = 2^log2_n keys of key_bytes
 * bytes (4: bitonic_sort_u32, 8: the composites of bitonic_sort_pairs_u32)
 * use opt's tile_log2, keys_per_thread_log2, global_bits and pipeline
 * instead of the process-wide values (the other fields are ignored).
 * opt == NULL removes the class's choice.  Written by the autotuner
 * (paper_1506_01446_gb300.autotune); BITONIC_ERR_UNSUPPORTED if the planner
 * rejects the choice for that class.
 */
bitonic_status bitonic_set_class_options(int key_bytes, int log2_n, const bitonic_options *opt);

/*
 * Describes the launch sequence bitonic_sort_u32 (pairs != 0: the composite
 * sort of bitonic_sort_pairs_u32) would run for n under the current options:
 * *launches = kernel launches, *hbm_passes = passes that read and write every
 * key once (the design's memory traffic is hbm_passes * 2 * N * key bytes),
 * *fused_steps and *global_steps = network steps done on chip / in global
 * passes.  Any output pointer may be NULL.
 */
bitonic_status bitonic_plan_info(size_t n, int pairs, int *launches, int *hbm_passes,
                                 int *fused_steps, int *global_steps);

/*
 * Kernels one graph-replayed bitonic_sort_u32 (pairs != 0:
 * bitonic_sort_pairs_u32) of n keys launches under the current options:
 * bitonic_plan_info's launches with every launch of a split run (option
 * split_log2) counted once per tile range, which the unsplit sequence of
 * bitonic_sort_u32_profiled does not have.  A key array off a 16-byte
 * boundary may add a launch.  BITONIC_ERR_INVALID for a NULL kernels.
 */
bitonic_status bitonic_graph_kernels(size_t n, int pairs, int *kernels);

/*
 * Same as bitonic_sort_u32 but launched without a graph, recording
 * events[i] on `stream` before launch i of the sequence and events[L] after
 * the last one (L = launches of bitonic_plan_info).  nevents must be >= L + 1.
 * kinds (may be NULL, >= L entries) receives each launch's kernel kind:
 * 0 = tile sort, 1 = global multi-stride pass, 2 = tile merge, 3 = single
 * step (basic variant).
 */
bitonic_status bitonic_sort_u32_profiled(uint32_t *keys, size_t n, int ascending,
                                         bitonic_stream_t stream, bitonic_event_t *events,
                                         int nevents, int *kinds);

/*
 * Copies the launch plan of an n-key sort (key_bytes 4: keys, 8: pair
 * composites) under the current options (with a size class's tuned options
 * where bitonic_set_class_options installed some), for inspection and host-side
 * tests.  info (max_info ints) receives N, the tile configuration id, its
 * log2 keys per thread and log2 threads per CTA, the launch count L and the
 * descriptor count D, then 7 ints per launch (kind, phase, hi, lo, flip,
 * descriptor index, grid).  descs receives D descriptors of
 * bitonic_debug_desc_size() bytes each (may be NULL).  Launches nothing.
 */
bitonic_status bitonic_debug_plan(size_t n, int key_bytes, int *info, int max_info, void *descs,
                                  int max_descs);
size_t bitonic_debug_desc_size(void);

/*
 * Key/value sort that allocates no device memory (the paper has no
 * counterpart; this is a deployment variant of bitonic_sort_pairs_u32).
 *
 * For callers that cannot let the library call cudaMalloc: applications
 * whose own memory manager owns all of the device memory and forbids
 * allocations behind its back, and latency-critical paths that cannot afford
 * cudaMalloc's implicit synchronisation with the device.  Same arguments,
 * ordering and result as bitonic_sort_pairs_u32, but the 64-bit composites
 * live in a fixed array of 2^20 entries (8 MiB) compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *   - n > 2^20 returns BITONIC_ERR_UNSUPPORTED without launching anything.
 *   - The first call on a device looks up the array's address and sets the
 *     kernels' shared-memory limit (no allocation); make that first call
 *     before any stream capture on the device.
 *   - All calls on a device share the one array, which keeps the last
 *     call's contents: calls whose work overlaps on the GPU (for instance on
 *     different streams) race and give wrong results.  Order them on one
 *     stream.
 *   - Launches go straight to `stream` (no cached graph), with the default
 *     tile configuration regardless of bitonic_set_options.
 */
bitonic_status bitonic_sort_pairs_u32_noalloc(uint32_t *keys, uint32_t *vals, size_t n, int ascending,
                                              bitonic_stream_t stream);

/*
 * Continuous-batching sort server (no paper counterpart; a deployment loop
 * around the sorts above).  bitonic_serve_run serves a whole stream of
 * requests on the calling host thread and returns when every request is
 * done:
 *   - Requests (reqs[0..nreq), arrival_s non-decreasing, seconds after the
 *     call's start) become pending when the host clock reaches their
 *     arrival.  Pending requests are admitted in arrival order while their
 *     device buffers fit cfg->dev_arena and their results fit the host
 *     output area (first fit in 16-byte units; a request that does not fit
 *     stops admission until a completion frees space).
 *   - Small requests (n <= small_keys keys-only, n <= small_pairs key/value)
 *     admitted in one pass are packed, at most max_batch per launch, into one
 *     bitonic_sort_segmented_u32 or bitonic_sort_segmented_pairs_u32_bounded
 *     launch per kind; a larger request gets its own bitonic_sort_u32 or
 *     bitonic_sort_pairs_u32.  Every request is sorted ascending (pairs: ties
 *     by index), exactly as sorted alone.
 *   - Each launch takes the next of cfg->streams in turn: its inputs are
 *     copied from the host pools, its segment offsets from cfg->offs_stage,
 *     its results back to out_keys / out_vals, all on that stream; an event
 *     marks it done, and the loop polls those events between admissions.
 *   - done_s[i] = the host time (seconds after the start) at which the loop
 *     saw request i's launch complete; out_pos[i] = the first key of its
 *     result in out_keys (and out_vals).  With keep_outputs == 0 result
 *     space is reused once the loop has seen a launch complete, so read
 *     results only with keep_outputs != 0 (then out_cap must hold every
 *     request's keys).
 *   - Graph replay is off for this thread during the call (plain launches;
 *     the thread's previous mode is restored).  Call the sorts once per
 *     stream beforehand for the sizes to come if no request should pay for
 *     workspace allocation or planning.
 *   - Ownership: every buffer is the caller's; host buffers should be page
 *     locked (the copies are asynchronous); dev_arena 16-byte aligned.
 *   - BITONIC_ERR_INVALID for a null or inconsistent argument, a request with
 *     n == 0, a source range outside the pools, or a request larger than the
 *     device arena or the output area (it could never be admitted).  A sort
 *     or CUDA error stops the loop: every stream is synchronised, the status
 *     is returned, and done_s of unfinished requests is negative.
 */
typedef struct {
    double arrival_s;   /* seconds after the start of the call */
    uint64_t src;       /* first key (and value) in in_keys / in_vals */
    uint32_t n;         /* keys, >= 1 */
    int32_t has_vals;   /* nonzero: a key/value request */
} bitonic_serve_request;

typedef struct {
    void *dev_arena;                  /* device memory the buffers are carved from */
    size_t dev_bytes;                 /* its size: the device memory budget */
    const uint32_t *in_keys;          /* input pools, pool_len entries each (host) */
    const uint32_t *in_vals;          /* may be NULL when no request has values */
    size_t pool_len;
    uint32_t *out_keys;               /* result area, out_cap entries each (host) */
    uint32_t *out_vals;               /* may be NULL when no request has values */
    size_t out_cap;
    int32_t *offs_stage;              /* staging for segment offsets, offs_cap entries (host) */
    size_t offs_cap;
    const bitonic_stream_t *streams;  /* launches go to these in turn */
    int nstreams;
    uint32_t small_keys;              /* packed keys-only requests: n <= small_keys (<= 16384) */
    uint32_t small_pairs;             /* packed key/value requests: n <= small_pairs (<= 8192) */
    int max_batch;                    /* most requests per packed launch (>= 1) */
    int keep_outputs;                 /* nonzero: result space is never reused */
} bitonic_serve_config;

typedef struct {
    double span_s;              /* first arrival to last completion */
    int64_t batches;            /* packed launches */
    int64_t batched_requests;   /* requests in packed launches */
    int64_t large_launches;     /* requests sorted alone */
    uint64_t peak_device_bytes; /* most of dev_arena in use at once */
} bitonic_serve_stats;

bitonic_status bitonic_serve_run(const bitonic_serve_config *cfg, const bitonic_serve_request *reqs, int nreq,
                                 double *done_s, uint64_t *out_pos, bitonic_serve_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* BITONIC_H */
