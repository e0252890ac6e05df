// Continuous-batching sort server: the loop behind bitonic_serve_run.
//
// One host thread admits requests as they arrive, carves their device
// buffers out of the caller's arena (first fit), packs small requests into
// segmented launches, spreads launches over the caller's streams and polls
// one event per launch for completion.  Every sort is one of the library's
// own entry points; this file only schedules copies and launches.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "bitonic.h"
#include "internal.h"

namespace bitonic {
namespace {

constexpr uint64_t kUnit = 16;  // allocation granule (bytes) of every arena

uint64_t round_unit(uint64_t bytes) { return (bytes + kUnit - 1) / kUnit * kUnit; }

// First-fit allocator over [0, size) bytes in kUnit granules; the free list
// is sorted by offset and coalesced on release.
class Arena {
public:
    explicit Arena(uint64_t size)
    {
        if (size >= kUnit) free_.push_back({0, size / kUnit * kUnit});
    }

    bool alloc(uint64_t bytes, uint64_t* off)
    {
        const uint64_t need = round_unit(bytes);
        for (size_t i = 0; i < free_.size(); ++i) {
            if (free_[i].len < need) continue;
            *off = free_[i].off;
            if (free_[i].len == need) {
                free_.erase(free_.begin() + (std::ptrdiff_t)i);
            } else {
                free_[i].off += need;
                free_[i].len -= need;
            }
            used_ += need;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }

    void release(uint64_t off, uint64_t bytes)
    {
        const uint64_t len = round_unit(bytes);
        used_ -= len;
        auto it = std::lower_bound(free_.begin(), free_.end(), off,
                                   [](const Block& b, uint64_t o) { return b.off < o; });
        it = free_.insert(it, {off, len});
        auto nx = it + 1;
        if (nx != free_.end() && it->off + it->len == nx->off) {
            it->len += nx->len;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = it - 1;
            if (pv->off + pv->len == it->off) {
                pv->len += it->len;
                free_.erase(it);
            }
        }
    }

    uint64_t peak() const { return peak_; }

private:
    struct Block {
        uint64_t off, len;
    };
    std::vector<Block> free_;
    uint64_t used_ = 0, peak_ = 0;
};

enum Kind { kSmallKeys = 0, kSmallPairs = 1, kLarge = 2 };

struct Flight {
    cudaEvent_t ev;
    std::vector<int> ids;
    uint64_t dev_off, dev_bytes;
    uint64_t host_off, host_bytes;
    uint64_t offs_off, offs_bytes;  // offs_bytes == 0: no staged offsets
};

// Restores the calling thread's graph mode on every way out.
struct GraphModeGuard {
    int prev;
    GraphModeGuard() : prev(thread_graph_mode()) { bitonic_set_thread_graphs(0); }
    ~GraphModeGuard() { bitonic_set_thread_graphs(prev); }
};

class Server {
public:
    Server(const bitonic_serve_config& c, const bitonic_serve_request* r, int n, double* done_s,
           uint64_t* out_pos)
        : c_(c), r_(r), n_(n), done_s_(done_s), out_pos_(out_pos), dev_(c.dev_bytes), host_(4 * c.out_cap),
          offs_(4 * c.offs_cap)
    {
    }

    ~Server()
    {
        for (cudaEvent_t e : events_) cudaEventDestroy(e);
    }

    bitonic_status run(bitonic_serve_stats* stats)
    {
        for (int i = 0; i < c_.nstreams; ++i)
            if (cudaStreamSynchronize((cudaStream_t)c_.streams[i]) != cudaSuccess)
                return report_error(BITONIC_ERR_CUDA, "bitonic_serve_run: stream synchronize");
        t0_ = std::chrono::steady_clock::now();
        int nxt = 0, done = 0;
        std::vector<int> pending, keep;
        while (done < n_) {
            const double now = elapsed();
            while (nxt < n_ && r_[nxt].arrival_s <= now) pending.push_back(nxt++);
            // admission in arrival order: small requests grouped per kind,
            // large ones alone; a request that does not fit stops admission
            std::vector<int> groups[2];
            keep.clear();
            bool blocked = false;
            for (int id : pending) {
                if (blocked) {
                    keep.push_back(id);
                    continue;
                }
                const Kind k = kind(id);
                if (k == kLarge) {
                    bool placed = false;
                    bitonic_status st = launch(std::vector<int>{id}, kLarge, &placed);
                    if (st != BITONIC_OK) return fail(st);
                    if (!placed) {
                        blocked = true;
                        keep.push_back(id);
                    } else {
                        ++large_;
                    }
                    continue;
                }
                std::vector<int>& g = groups[k];
                g.push_back(id);
                if ((int)g.size() == c_.max_batch) {
                    bitonic_status st = launch_group(g, k, keep, &blocked);
                    if (st != BITONIC_OK) return fail(st);
                    g.clear();
                }
            }
            for (int k = 0; k < 2; ++k) {
                std::vector<int>& g = groups[k];
                if (g.empty()) continue;
                if (blocked) {
                    keep.insert(keep.end(), g.begin(), g.end());
                    continue;
                }
                bitonic_status st = launch_group(g, (Kind)k, keep, &blocked);
                if (st != BITONIC_OK) return fail(st);
            }
            std::sort(keep.begin(), keep.end());
            pending.swap(keep);
            // completions
            int finished = 0;
            bitonic_status st = poll(&finished);
            if (st != BITONIC_OK) return fail(st);
            done += finished;
            if (pending.empty() && inflight_.empty() && nxt < n_) {
                const double wait = r_[nxt].arrival_s - elapsed();
                if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 1e-4));
            }
        }
        if (stats) {
            double last = 0.0, first = n_ ? r_[0].arrival_s : 0.0;
            for (int i = 0; i < n_; ++i) last = std::max(last, done_s_[i]);
            stats->span_s = last - first;
            stats->batches = batches_;
            stats->batched_requests = batched_;
            stats->large_launches = large_;
            stats->peak_device_bytes = dev_.peak();
        }
        return BITONIC_OK;
    }

private:
    double elapsed() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0_).count();
    }

    Kind kind(int id) const
    {
        const bitonic_serve_request& q = r_[id];
        if (q.has_vals) return q.n <= c_.small_pairs ? kSmallPairs : kLarge;
        return q.n <= c_.small_keys ? kSmallKeys : kLarge;
    }

    // Launches a packed group; if it does not fit while nothing is in flight
    // (so it never would), its first half goes alone (recursively) and the
    // rest waits.  Requests not launched go to keep and block admission.
    bitonic_status launch_group(const std::vector<int>& g, Kind k, std::vector<int>& keep, bool* blocked)
    {
        bool placed = false;
        bitonic_status st = launch(g, k, &placed);
        if (st != BITONIC_OK) return st;
        if (placed) {
            ++batches_;
            batched_ += (int64_t)g.size();
            return BITONIC_OK;
        }
        if (inflight_.empty() && g.size() > 1) {
            const size_t h = g.size() / 2;
            std::vector<int> head(g.begin(), g.begin() + (std::ptrdiff_t)h);
            st = launch_group(head, k, keep, blocked);
            if (st != BITONIC_OK) return st;
            keep.insert(keep.end(), g.begin() + (std::ptrdiff_t)h, g.end());
        } else {
            keep.insert(keep.end(), g.begin(), g.end());
        }
        *blocked = true;
        return BITONIC_OK;
    }

    // Allocates, copies in, sorts, copies out and records the launch's event;
    // *placed = false (and nothing enqueued) if a buffer does not fit.
    bitonic_status launch(const std::vector<int>& ids, Kind k, bool* placed)
    {
        *placed = false;
        uint64_t total = 0;
        for (int id : ids) total += r_[id].n;
        const bool pairs = k == kSmallPairs || (k == kLarge && r_[ids[0]].has_vals);
        const bool batch = k != kLarge;
        const uint64_t kbytes = round_unit(4 * total);
        const uint64_t dev_bytes = kbytes * (pairs ? 2 : 1) + (batch ? 4 * (ids.size() + 1) : 0);
        Flight f{};
        f.dev_bytes = dev_bytes;
        f.host_bytes = 4 * total;
        f.offs_bytes = batch ? 4 * (ids.size() + 1) : 0;
        if (!dev_.alloc(f.dev_bytes, &f.dev_off)) return BITONIC_OK;
        if (!host_.alloc(f.host_bytes, &f.host_off)) {
            dev_.release(f.dev_off, f.dev_bytes);
            return BITONIC_OK;
        }
        if (batch && !offs_.alloc(f.offs_bytes, &f.offs_off)) {
            dev_.release(f.dev_off, f.dev_bytes);
            host_.release(f.host_off, f.host_bytes);
            return BITONIC_OK;
        }
        *placed = true;
        f.ids = ids;
        cudaStream_t s = (cudaStream_t)c_.streams[rr_++ % c_.nstreams];
        unsigned char* base = static_cast<unsigned char*>(c_.dev_arena) + f.dev_off;
        uint32_t* dk = reinterpret_cast<uint32_t*>(base);
        uint32_t* dv = pairs ? reinterpret_cast<uint32_t*>(base + kbytes) : nullptr;
        // inputs: one copy per run of consecutive sources
        uint64_t pos = 0;
        for (size_t i = 0; i < ids.size();) {
            size_t j = i + 1;
            uint64_t n = r_[ids[i]].n;
            while (j < ids.size() && r_[ids[j]].src == r_[ids[j - 1]].src + r_[ids[j - 1]].n) n += r_[ids[j++]].n;
            const uint64_t src = r_[ids[i]].src;
            if (cudaMemcpyAsync(dk + pos, c_.in_keys + src, 4 * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                (pairs && cudaMemcpyAsync(dv + pos, c_.in_vals + src, 4 * n, cudaMemcpyHostToDevice, s) != cudaSuccess))
                return release_failed(f, "bitonic_serve_run: input copy");
            pos += n;
            i = j;
        }
        bitonic_status st;
        if (batch) {
            int32_t* stage = c_.offs_stage + f.offs_off / 4;
            int32_t* doffs = reinterpret_cast<int32_t*>(base + kbytes * (pairs ? 2 : 1));
            stage[0] = 0;
            for (size_t q = 0; q < ids.size(); ++q) stage[q + 1] = stage[q] + (int32_t)r_[ids[q]].n;
            if (cudaMemcpyAsync(doffs, stage, f.offs_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return release_failed(f, "bitonic_serve_run: offsets copy");
            st = pairs ? bitonic_sort_segmented_pairs_u32_bounded(dk, dv, doffs, (int)ids.size(), (int)c_.small_pairs,
                                                                   (bitonic_stream_t)s)
                       : bitonic_sort_segmented_u32(dk, doffs, (int)ids.size(), (bitonic_stream_t)s);
        } else {
            st = pairs ? bitonic_sort_pairs_u32(dk, dv, total, 1, (bitonic_stream_t)s)
                       : bitonic_sort_u32(dk, total, 1, (bitonic_stream_t)s);
        }
        if (st != BITONIC_OK) {
            inflight_.push_back(f);  // its copies may be in flight: freed after the streams drain
            return st;
        }
        const uint64_t hk = f.host_off / 4;
        if (cudaMemcpyAsync(c_.out_keys + hk, dk, 4 * total, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            (pairs && cudaMemcpyAsync(c_.out_vals + hk, dv, 4 * total, cudaMemcpyDeviceToHost, s) != cudaSuccess))
            return release_failed(f, "bitonic_serve_run: result copy");
        if (events_free_.empty()) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                return release_failed(f, "bitonic_serve_run: event create");
            events_.push_back(e);
            events_free_.push_back(e);
        }
        f.ev = events_free_.back();
        events_free_.pop_back();
        if (cudaEventRecord(f.ev, s) != cudaSuccess) return release_failed(f, "bitonic_serve_run: event record");
        uint64_t p = hk;
        for (int id : ids) {
            out_pos_[id] = p;
            p += r_[id].n;
        }
        inflight_.push_back(f);
        return BITONIC_OK;
    }

    bitonic_status release_failed(const Flight& f, const char* what)
    {
        inflight_.push_back(f);
        return report_error(BITONIC_ERR_CUDA, what);
    }

    bitonic_status poll(int* finished)
    {
        size_t w = 0;
        for (size_t i = 0; i < inflight_.size(); ++i) {
            Flight& f = inflight_[i];
            const cudaError_t q = cudaEventQuery(f.ev);
            if (q == cudaErrorNotReady) {
                inflight_[w++] = f;
                continue;
            }
            if (q != cudaSuccess) return report_error(BITONIC_ERR_CUDA, "bitonic_serve_run: event query");
            const double t = elapsed();
            for (int id : f.ids) done_s_[id] = t;
            *finished += (int)f.ids.size();
            dev_.release(f.dev_off, f.dev_bytes);
            if (!c_.keep_outputs) host_.release(f.host_off, f.host_bytes);
            if (f.offs_bytes) offs_.release(f.offs_off, f.offs_bytes);
            events_free_.push_back(f.ev);
        }
        inflight_.resize(w);
        return BITONIC_OK;
    }

    // After an error: drain the streams so that no copy still uses the
    // caller's buffers, then return the status.
    bitonic_status fail(bitonic_status st)
    {
        for (int i = 0; i < c_.nstreams; ++i) cudaStreamSynchronize((cudaStream_t)c_.streams[i]);
        return st;
    }

    const bitonic_serve_config& c_;
    const bitonic_serve_request* r_;
    int n_;
    double* done_s_;
    uint64_t* out_pos_;
    Arena dev_, host_, offs_;
    std::vector<Flight> inflight_;
    std::vector<cudaEvent_t> events_, events_free_;
    std::chrono::steady_clock::time_point t0_;
    int rr_ = 0;
    int64_t batches_ = 0, batched_ = 0, large_ = 0;
};

bitonic_status check_config(const bitonic_serve_config* c, const bitonic_serve_request* reqs, int nreq,
                            const double* done_s, const uint64_t* out_pos)
{
    if (!c || nreq < 0 || (nreq > 0 && (!reqs || !done_s || !out_pos)))
        return report_error(BITONIC_ERR_INVALID, "bitonic_serve_run: null argument");
    if (nreq == 0) return BITONIC_OK;
    if (!c->dev_arena || ((uintptr_t)c->dev_arena & 15u) || !c->in_keys || !c->out_keys || !c->offs_stage ||
        !c->streams || c->nstreams < 1 || c->max_batch < 1 || c->small_keys > 16384 || c->small_pairs > 8192)
        return report_error(BITONIC_ERR_INVALID, "bitonic_serve_run: bad configuration");
    uint64_t all_keys = 0;
    for (int i = 0; i < nreq; ++i) {
        const bitonic_serve_request& q = reqs[i];
        if (q.n == 0 || q.src > c->pool_len || q.n > c->pool_len - q.src || (i && q.arrival_s < reqs[i - 1].arrival_s))
            return report_error(BITONIC_ERR_INVALID, "bitonic_serve_run: bad request " + std::to_string(i));
        if (q.has_vals && (!c->in_vals || !c->out_vals))
            return report_error(BITONIC_ERR_INVALID, "bitonic_serve_run: values without value buffers");
        const bool small = q.has_vals ? q.n <= c->small_pairs : q.n <= c->small_keys;
        const uint64_t dev = round_unit(4ull * q.n) * (q.has_vals ? 2 : 1) + (small ? 8 : 0);
        if (dev > c->dev_bytes || 4ull * q.n > 4ull * c->out_cap || (small && c->offs_cap < 2))
            return report_error(BITONIC_ERR_INVALID,
                                "bitonic_serve_run: request " + std::to_string(i) + " can never be admitted");
        all_keys += round_unit(4ull * q.n) / 4;
    }
    if (c->keep_outputs && all_keys > c->out_cap)
        return report_error(BITONIC_ERR_INVALID, "bitonic_serve_run: keep_outputs needs every result in out_keys");
    return BITONIC_OK;
}

}  // namespace
}  // namespace bitonic

using namespace bitonic;

extern "C" bitonic_status bitonic_serve_run(const bitonic_serve_config* cfg, const bitonic_serve_request* reqs,
                                            int nreq, double* done_s, uint64_t* out_pos, bitonic_serve_stats* stats)
{
    bitonic_status st = check_config(cfg, reqs, nreq, done_s, out_pos);
    if (st != BITONIC_OK) return st;
    for (int i = 0; i < nreq; ++i) {
        done_s[i] = -1.0;
        out_pos[i] = 0;
    }
    if (stats) *stats = bitonic_serve_stats{};
    if (nreq == 0) return BITONIC_OK;
    GraphModeGuard guard;
    Server srv(*cfg, reqs, nreq, done_s, out_pos);
    return srv.run(stats);
}
