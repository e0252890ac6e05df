// Host planner: turns a sort of n keys into a launch sequence and builds the
// tile descriptors (global mapping + register rounds) of every launch.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "desc.h"
#include "internal.h"
#include "kernel_cfg.h"
#include "patterns.h"

namespace bitonic {

namespace {

constexpr TileCfg cfg_row(int id)
{
#define BITONIC_CFG_ROW(ID, KT, LR, LT, MB) \
    if (id == ID) return TileCfg{ID, (int)sizeof(KT), LR, LT, MB};
    BITONIC_TILE_CONFIGS(BITONIC_CFG_ROW)
#undef BITONIC_CFG_ROW
    return TileCfg{-1, 0, 0, 0, 0};
}

const TileCfg kCfgs[kNumTileCfgs] = {cfg_row(0), cfg_row(1), cfg_row(2), cfg_row(3), cfg_row(4),
                                     cfg_row(5), cfg_row(6), cfg_row(7), cfg_row(8)};

struct LStep {
    int bit;
    bool flip;
};

// Phases 1..kmax of the network on local bits (Section 3.1): phase q starts
// with the mirror step at bit q-1, then half-cleaners at bits q-2..0.
std::vector<LStep> tile_sort_steps(int kmax)
{
    std::vector<LStep> s;
    for (int q = 1; q <= kmax; ++q) {
        s.push_back({q - 1, true});
        for (int b = q - 2; b >= 0; --b) s.push_back({b, false});
    }
    return s;
}

bool contains(const std::vector<int>& v, int x) { return std::find(v.begin(), v.end(), x) != v.end(); }

// Thread-bit order: lanes 0..2 on local vector bits of distinct residue mod 3
// (conflict-free 16-byte shared accesses under the swizzle), smallest first,
// then the rest ascending.
std::vector<int> order_thread_bits(const std::vector<int>& T, int vb)
{
    std::vector<int> out;
    bool used[3] = {false, false, false};
    for (int pick = 0; pick < 3; ++pick) {
        for (int b : T) {
            if (contains(out, b)) continue;
            const int res = (b - vb) % 3;
            if (used[res]) continue;
            out.push_back(b);
            used[res] = true;
            break;
        }
    }
    for (int b : T)
        if (!contains(out, b)) out.push_back(b);
    return out;
}

// Local bits in [vb, bit) that are thread bits when R are the register bits.
uint32_t mirror_mask(int bit, const std::vector<int>& R, int vb)
{
    uint32_t mask = 0;
    for (int b = vb; b < bit; ++b)
        if (!contains(R, b)) mask |= 1u << b;
    return mask;
}

struct HostRound {
    std::vector<int> R;          // register bits (ascending), local bits >= vb
    std::vector<LStep> steps;
    int mirror_bit = -1;         // register bit carrying thread components
    uint32_t mirror = 0;
};

void fill_registers(std::vector<int>& R, int RR, int m, int vb)
{
    for (int b = m - 1; b >= vb && (int)R.size() < RR; --b)
        if (!contains(R, b)) R.push_back(b);
    std::sort(R.begin(), R.end());
}

bool build_round(const std::vector<LStep>& steps, size_t i, size_t& j, int RR, int m, int vb, HostRound& hr)
{
    // Greedy: take steps while their bits fit in the register budget.
    std::vector<int> R;
    j = i;
    while (j < steps.size()) {
        const int b = steps[j].bit;
        if (b >= vb && !contains(R, b)) {
            if ((int)R.size() == RR) break;
            R.push_back(b);
        }
        ++j;
    }
    // A mirror step whose lower bits include thread bits must be the last
    // mirror step of its round, and its bit may not be used again there.
    for (;;) {
        R.clear();
        for (size_t s = i; s < j; ++s)
            if (steps[s].bit >= vb && !contains(R, steps[s].bit)) R.push_back(steps[s].bit);
        fill_registers(R, RR, m, vb);
        size_t bad = j;
        int mbit = -1;
        for (size_t s = i; s < j; ++s) {
            if (steps[s].flip) {
                if (mbit >= 0) { bad = s; break; }
                if (mirror_mask(steps[s].bit, R, vb)) mbit = steps[s].bit;
            } else if (mbit >= 0 && steps[s].bit == mbit) {
                bad = s;
                break;
            }
        }
        if (bad == j) {
            hr.R = R;
            hr.steps.assign(steps.begin() + i, steps.begin() + j);
            hr.mirror_bit = mbit;
            hr.mirror = mbit >= 0 ? mirror_mask(mbit, R, vb) : 0;
            return true;
        }
        if (bad <= i) return false;
        j = bad;
    }
}

// Thread bits of a round: the local bits at or above vb that are not
// register bits.
std::vector<int> thread_bits(const HostRound& hr, int m, int vb)
{
    std::vector<int> T;
    for (int b = vb; b < m; ++b)
        if (!contains(hr.R, b)) T.push_back(b);
    return T;
}

// Descriptor of round hr with thread-index bit i on local bit T[i].
bool emit_round_ordered(const HostRound& hr, const std::vector<int>& T, int log_t, int m, int vb, RoundDesc& rd)
{
    std::memset(&rd, 0, sizeof(rd));
    if ((int)T.size() != log_t) return false;
    for (int t = 0; t < log_t; ++t) rd.thr_loc[t] = (uint16_t)(1u << T[t]);
    for (size_t q = 0; q < hr.R.size(); ++q) {
        uint32_t v = 1u << hr.R[q];
        if (hr.R[q] == hr.mirror_bit) v |= hr.mirror;
        rd.reg_loc[q] = (uint16_t)v;
    }
    // 16-byte vector slots as byte offsets (m - vb <= 12 slot bits: below 64 KiB)
    if (m - vb > 12) return false;
    for (int t = 0; t < log_t; ++t) rd.thr_sw[t] = (uint16_t)(smem_swizzle(rd.thr_loc[t] >> vb) << 4);
    for (size_t q = 0; q < hr.R.size(); ++q) rd.reg_sw[q] = (uint16_t)(smem_swizzle(rd.reg_loc[q] >> vb) << 4);
    if (hr.steps.size() > (size_t)kMaxStepsPerRound) return false;
    rd.nsteps = (uint8_t)hr.steps.size();
    for (size_t s = 0; s < hr.steps.size(); ++s) {
        const int b = hr.steps[s].bit;
        int q;
        if (b < vb) {
            q = b;
        } else {
            q = vb + (int)(std::find(hr.R.begin(), hr.R.end(), b) - hr.R.begin());
        }
        rd.steps[s] = (uint8_t)(q | (hr.steps[s].flip ? kStepFlip : 0));
    }
    return true;
}

bool emit_round(const HostRound& hr, int log_t, int m, int vb, RoundDesc& rd)
{
    return emit_round_ordered(hr, order_thread_bits(thread_bits(hr, m, vb), vb), log_t, m, vb, rd);
}

// Lanes 0..2 on local bits vb..vb+2 that the map sends to global units:
// each quarter warp then touches one aligned 128-byte line.
bool round_coalesced(const RoundDesc& rd, const TileParamsBig& P, int vb)
{
    const int need = std::min(3, (int)P.row_log - vb);  // lanes that stay inside one row
    for (int t = 0; t < need; ++t) {
        const int b = vb + t;
        if (rd.thr_loc[t] != (1u << b)) return false;
        if (P.gvec[b] != (1u << b)) return false;
    }
    return true;
}

HostRound io_round(int RR, int m, int vb)
{
    HostRound hr;
    for (int b = m - 1; b >= vb + 3 && (int)hr.R.size() < RR; --b) hr.R.push_back(b);
    std::sort(hr.R.begin(), hr.R.end());
    return hr;
}

uint32_t global_of_local(const TileParamsBig& P, uint32_t L)
{
    uint32_t g = 0;
    for (int j = 0; j < P.m; ++j)
        if ((L >> j) & 1u) g ^= P.gvec[j];
    return g;
}

void fill_io(const RoundDesc& rd, const TileParamsBig& P, int log_t, int nreg, IoDesc& io)
{
    std::memset(&io, 0, sizeof(io));
    for (int i = 0; i < log_t; ++i) io.thr_glob[i] = global_of_local(P, rd.thr_loc[i]);
    for (int j = 0; j < nreg; ++j) io.reg_glob[j] = global_of_local(P, rd.reg_loc[j]);
}

// Index of the catalog pattern whose steps equal the round's, else generic.
uint8_t find_pattern(const RoundDesc& rd, int log_r)
{
    const int n = catalog_size(log_r);
    for (int i = 0; i < n; ++i) {
        const RoundPattern p = catalog_pattern(log_r, i);
        if (p.n != rd.nsteps) continue;
        bool same = true;
        for (int s = 0; s < p.n; ++s) same &= p.steps[s] == rd.steps[s];
        if (same) return (uint8_t)i;
    }
    return kGenericPattern;
}

// Lanes per warp: thread-index bits 0..4.
constexpr int kLaneBits = 5;

// Canonical form of the shared-memory slots one warp touches in a round's
// layout: the reduced echelon basis of the span of the local vectors inside
// a warp (vector components, register bits, lanes), followed by each warp
// bit's local vector reduced modulo that span.  Two rounds with equal keys
// give every warp the same set of local indices, hence of slots.
std::vector<uint32_t> warp_key(const RoundDesc& rd, int log_t, int nreg, int vb)
{
    std::vector<uint32_t> basis;  // one vector per pivot (its highest bit), kept reduced
    auto reduce = [&](uint32_t v) {
        for (uint32_t b : basis) {
            const uint32_t top = 1u << (31 - __builtin_clz(b));
            if (v & top) v ^= b;
        }
        return v;
    };
    auto insert = [&](uint32_t v) {
        v = reduce(v);
        if (!v) return;
        const uint32_t top = 1u << (31 - __builtin_clz(v));
        for (uint32_t& b : basis)
            if (b & top) b ^= v;
        basis.push_back(v);
        std::sort(basis.begin(), basis.end());
    };
    for (int c = 0; c < vb; ++c) insert(1u << c);
    for (int j = 0; j < nreg; ++j) insert(rd.reg_loc[j]);
    for (int t = 0; t < std::min(kLaneBits, log_t); ++t) insert(rd.thr_loc[t]);
    std::vector<uint32_t> key = basis;
    for (int t = kLaneBits; t < log_t; ++t) key.push_back(reduce(rd.thr_loc[t]) | 0x80000000u);
    return key;
}

// Chooses every round's thread-bit order (which non-register bits are lanes
// and which select the warp) so that as many transposes as possible keep
// each warp's slots, then marks those rounds warp-local.  Lanes 0..2 keep
// local bits of distinct residue mod 3 (conflict-free 16-byte shared
// accesses); a first or last round that is coalesced stays coalesced.  A
// dynamic program over the rounds: score 2 per warp-local transpose, 1 per
// round left in its default order.
bool choose_thread_orders(const std::vector<HostRound>& hrs, std::vector<RoundDesc>& out, const TileParamsBig& P,
                          int log_t, int m, int vb, int nreg)
{
    const size_t nr = out.size();
    if (nr < 2 || log_t <= kLaneBits) return true;
    const int nwarp = log_t - kLaneBits;
    struct Cand {
        RoundDesc rd;
        std::vector<uint32_t> key;
        int score = 0;
        int prev = -1;
    };
    std::vector<std::vector<Cand>> cands(nr);
    for (size_t r = 0; r < nr; ++r) {
        const std::vector<int> T = thread_bits(hrs[r], m, vb);
        if ((int)T.size() != log_t) return false;
        const bool keep_coalesced = (r == 0 || r + 1 == nr) && round_coalesced(out[r], P, vb);
        Cand def;
        def.rd = out[r];
        def.key = warp_key(out[r], log_t, nreg, vb);
        def.score = 1;
        cands[r].push_back(def);
        // every choice of the warp bits among the thread bits
        const int nt = (int)T.size();
        for (uint32_t sel = 0; sel < (1u << nt); ++sel) {
            if (__builtin_popcount(sel) != nwarp) continue;
            std::vector<int> lanes, warps;
            for (int t = 0; t < nt; ++t) ((sel >> t) & 1u ? warps : lanes).push_back(T[t]);
            std::vector<int> order = order_thread_bits(lanes, vb);
            bool res[3] = {false, false, false};
            for (int t = 0; t < 3; ++t) res[(order[t] - vb) % 3] = true;
            if (!(res[0] && res[1] && res[2])) continue;
            order.insert(order.end(), warps.begin(), warps.end());
            Cand c;
            if (!emit_round_ordered(hrs[r], order, log_t, m, vb, c.rd)) return false;
            if (keep_coalesced && !round_coalesced(c.rd, P, vb)) continue;
            if (std::memcmp(&c.rd, &out[r], sizeof(RoundDesc)) == 0) continue;  // the default
            c.key = warp_key(c.rd, log_t, nreg, vb);
            cands[r].push_back(c);
        }
    }
    for (size_t r = 1; r < nr; ++r)
        for (Cand& c : cands[r]) {
            int best = -1, arg = -1;
            for (size_t q = 0; q < cands[r - 1].size(); ++q) {
                const Cand& p = cands[r - 1][q];
                const int v = p.score + (p.key == c.key ? 2 : 0);
                if (v > best) { best = v; arg = (int)q; }
            }
            c.score += best;
            c.prev = arg;
        }
    int arg = 0;
    for (size_t q = 1; q < cands[nr - 1].size(); ++q)
        if (cands[nr - 1][q].score > cands[nr - 1][arg].score) arg = (int)q;
    for (size_t r = nr; r-- > 0;) {
        const Cand& c = cands[r][arg];
        out[r] = c.rd;
        if (r > 0) {
            out[r].warp_local = cands[r - 1][c.prev].key == c.key ? 1 : 0;
            arg = c.prev;
        }
    }
    return true;
}

bool plan_rounds(const std::vector<LStep>& steps, const TileCfg& cfg, int vb, int io_direct, TileParamsBig& P,
                 bool warp_sync = false)
{
    const int m = cfg.log_r + cfg.log_t;
    const int RR = cfg.log_r - vb;
    std::vector<HostRound> rounds;
    size_t i = 0;
    while (i < steps.size()) {
        size_t j;
        HostRound hr;
        if (!build_round(steps, i, j, RR, m, vb, hr)) return false;
        rounds.push_back(hr);
        i = j;
    }
    if (rounds.empty()) rounds.push_back(io_round(RR, m, vb));
    std::vector<RoundDesc> out;
    for (auto& hr : rounds) {
        RoundDesc rd;
        if (!emit_round(hr, cfg.log_t, m, vb, rd)) return false;
        out.push_back(rd);
    }
    // Global loads and stores go through a coalesced layout: add a round
    // without steps (one more shared-memory transpose) where needed.
    RoundDesc io;
    const HostRound ioh = io_round(RR, m, vb);
    if (!emit_round(ioh, cfg.log_t, m, vb, io)) return false;
    if (!(io_direct & 1) && !round_coalesced(out.front(), P, vb)) {
        out.insert(out.begin(), io);
        rounds.insert(rounds.begin(), ioh);
    }
    if (!(io_direct & 2) && !round_coalesced(out.back(), P, vb)) {
        out.push_back(io);
        rounds.push_back(ioh);
    }
    if (out.size() > (size_t)kMaxRoundsBig) return false;
    if (warp_sync && !choose_thread_orders(rounds, out, P, cfg.log_t, m, vb, RR)) return false;
    for (RoundDesc& rd : out) rd.pattern = find_pattern(rd, cfg.log_r);
    P.nrounds = (uint8_t)out.size();
    for (size_t r = 0; r < out.size(); ++r) P.rounds[r] = out[r];
    fill_io(out.front(), P, cfg.log_t, RR, P.io[0]);
    fill_io(out.back(), P, cfg.log_t, RR, P.io[1]);
    return true;
}

// Tile over global bits B (ascending, m of them).  With affine_top, the top
// local bit carries a phase's mirror step: it maps to 2^top XOR every global
// bit below top that the tile leaves out.  The CTA index fills the other
// global bits below k, lowest first, as runs of consecutive bits.
bool map_bits(TileParamsBig& P, const std::vector<int>& B, bool affine_top, int k)
{
    const int m = (int)B.size();
    P.m = (uint8_t)m;
    for (int j = 0; j < m; ++j) P.gvec[j] = 1u << B[j];
    if (affine_top) {
        uint32_t v = 1u << B[m - 1];
        for (int b = 0; b < B[m - 1]; ++b)
            if (!contains(B, b)) v |= 1u << b;
        P.gvec[m - 1] = v;
    }
    P.contiguous = 1;
    for (int j = 0; j < m; ++j)
        if (B[j] != j) P.contiguous = 0;
    int c = 0;
    while (c < m && P.gvec[c] == (1u << c)) ++c;
    P.row_log = (uint8_t)c;
    P.span_mask = 0;
    for (int j = 0; j < m; ++j) P.span_mask |= P.gvec[j];
    int nr = 0;
    for (int b = 0; b < k;) {
        if (contains(B, b)) { ++b; continue; }
        int w = 0;
        while (b + w < k && !contains(B, b + w)) ++w;
        if (nr == kMaxCtaRuns) return false;
        P.run_shift[nr] = (uint8_t)b;
        P.run_width[nr] = (uint8_t)w;
        ++nr;
        b += w;
    }
    P.nruns = (uint8_t)nr;
    return true;
}

// Tile configuration for a sort of key_bytes keys: the semi variant uses
// the configurations with one register bit beyond the vector; otherwise the
// requested tile size and keys per thread (0 = default: 16K keys of 4 bytes,
// 8K composites of 8 bytes, 64 / 32 keys per thread).
int choose_cfg(int key_bytes, const Options& opt)
{
    const int vb = key_bytes == 4 ? 2 : 1;
    const bool semi = opt.variant == 2;
    const int tile = opt.tile_log2 ? opt.tile_log2 : (key_bytes == 4 ? 14 : 13);
    // Default keys per thread: 64 for 4-byte keys, 32 for composites, else
    // the largest configured value below that.
    const int pref_r = opt.keys_per_thread_log2 ? opt.keys_per_thread_log2 : (key_bytes == 4 ? 6 : 5);
    // Register cap: 3 = kernels capped for three resident CTAs per SM, 2 =
    // kernels bounded for two; 0 = automatic: two.  Measured on GB300 with the
    // shared-memory slots precomputed by the planner: 2^28 4-byte keys 12.54
    // against 12.73 ms, 2^22 0.169 against 0.180 ms (three CTAs win only
    // where the keys fit in L2: 2^24 0.647 against 0.631 ms); 2^26 pairs 8.79
    // against 9.47 ms.  A cap is taken where a capped kernel of this shape
    // exists; other shapes fall back to the two-CTA kernel.
    const int cap = opt.ctas_per_sm ? opt.ctas_per_sm : 2;
    const int want_blocks = cap == 3 ? 3 : 1;
    for (int blocks : {want_blocks, 1}) {
        int best = -1;
        for (int i = 0; i < kNumTileCfgs; ++i) {
            const TileCfg& c = kCfgs[i];
            if (c.key_bytes != key_bytes) continue;
            const bool c_semi = c.log_r == vb + 1;
            if (semi != c_semi) continue;
            if (semi) return i;
            if (c.log_r + c.log_t != tile) continue;
            if (opt.keys_per_thread_log2 && c.log_r != opt.keys_per_thread_log2) continue;
            if (c.log_r > pref_r) continue;
            if ((c.min_blocks == 3) != (blocks == 3)) continue;
            if (best < 0 || c.log_r > kCfgs[best].log_r) best = i;
        }
        if (best >= 0) return best;
    }
    return -1;
}

// Relative cost of one more pass (a full read and write of the keys) against
// one more shared-memory transpose inside a pass, measured on GB300 at
// 2^28 keys: about 0.30 ms against 0.075 ms.
#ifndef BITONIC_PASS_WEIGHT
#define BITONIC_PASS_WEIGHT 4
#endif
constexpr int kPassWeight = BITONIC_PASS_WEIGHT;

struct GStep {
    int bit;
    bool flip;
    int phase;
};

bool to_small(const TileParamsBig& b, TileParams& s)
{
    std::memset(&s, 0, sizeof(s));
    if (b.nrounds > kMaxRoundsSmall) return false;
    std::memcpy(&s, &b, offsetof(TileParamsBig, rounds));
    std::memcpy(s.rounds, b.rounds, b.nrounds * sizeof(RoundDesc));
    return true;
}

}  // namespace

const TileCfg& tile_cfg(int id) { return kCfgs[id]; }

// Descriptor of a packed segmented tile whose segments are padded to 2^k
// positions: phases 1..k of the network on a contiguous tile (16K or 8K
// keys, or 8K composites for pairs).
bool make_class_desc(int key_bytes, int k, TileParamsBig& P, int tile_log2)
{
    std::memset(&P, 0, sizeof(P));
    // the packed segmented kernels: 16K keys (256 x 64) or 8K keys (256 x 32);
    // 8K composites (256 x 32)
    const int cfg_id = key_bytes == 4 ? (tile_log2 == 13 ? 1 : 0) : 4;
    const TileCfg& cfg = kCfgs[cfg_id];
    const int vb = key_bytes == 4 ? 2 : 1;
    const int m = cfg.log_r + cfg.log_t;
    if (k < 1 || k > m) return false;
    std::vector<int> B;
    for (int b = 0; b < m; ++b) B.push_back(b);
    if (!map_bits(P, B, false, m)) return false;
    return plan_rounds(tile_sort_steps(k), cfg, vb, 0, P, true);
}

Plan make_plan(uint64_t nv, int key_bytes, const Options& opt)
{
    Plan plan;
    uint64_t N = 2;
    int k = 1;
    while (N < nv) { N <<= 1; ++k; }
    plan.N = N;
    plan.k = k;
    if (opt.variant == 1) {  // basic: one launch per step (Section 3.3)
        for (int p = 1; p <= k; ++p)
            for (int j = p - 1; j >= 0; --j)
                plan.launches.push_back({KIND_STEP, p, j, j, j == p - 1, -1, 0, false});
        plan.hbm_passes = (int)plan.launches.size();
        plan.global_steps = (int)plan.launches.size();
        plan.cfg = -1;
        plan.ok = true;
        return plan;
    }
    const int cfg_id = choose_cfg(key_bytes, opt);
    if (cfg_id < 0) return plan;
    const TileCfg& cfg = kCfgs[cfg_id];
    const int vb = key_bytes == 4 ? 2 : 1;
    const int m = cfg.log_r + cfg.log_t;
    // rows of at least 128 bytes by default (one line per quarter warp)
    const int c_min = opt.min_row_log2 ? std::max(vb + 1, opt.min_row_log2) : vb + 3;
    const bool semi = opt.variant == 2;
    const bool fuse = !semi;   // let a pass run across a phase boundary
    // Transposes that keep every warp's slots wait at a warp barrier (the
    // semi variant keeps a CTA barrier after every transpose).
    const bool warp_sync = !semi && opt.round_sync == 0;
    // At most this many strides at or above the tile size per pass; 0 =
    // automatic: 8 (2^28 4-byte keys on GB300: 13.34 ms against 13.59 ms
    // uncapped, the cost-based split then preferring 2-round passes).
    int high_limit = semi ? 1 : (opt.global_bits > 0 ? opt.global_bits : 8);
    plan.cfg = cfg_id;
    plan.tile_log2 = m;
    const uint32_t grid = k > m ? (1u << (k - m)) : 1u;

    auto add_pass = [&](const std::vector<int>& B, bool affine, const std::vector<LStep>& ls, int kind,
                        int phase, int hi, int lo, bool flip) -> bool {
        TileParamsBig P;
        std::memset(&P, 0, sizeof(P));
        if (!map_bits(P, B, affine, k)) return false;
        if (!plan_rounds(ls, cfg, vb, opt.io_direct, P, warp_sync)) return false;
        TileParams small;
        const bool fits = to_small(P, small);
        plan.descs.push_back(P);
        plan.small.push_back(small);
        plan.launches.push_back({kind, phase, hi, lo, flip ? 1 : 0, (int)plan.descs.size() - 1, grid, fits});
        plan.hbm_passes += 1;
        return true;
    };

    // Phases 1..min(k, m) of every tile on chip.
    const int ksort = std::min(k, m);
    {
        std::vector<int> B;
        for (int b = 0; b < m; ++b) B.push_back(b);
        if (!add_pass(B, false, tile_sort_steps(ksort), KIND_TILE_SORT, ksort, ksort - 1, 0, true)) return plan;
        plan.fused_steps += ksort * (ksort + 1) / 2;
    }

    // The remaining steps, split into passes.  A pass takes a run of steps
    // whose bits (plus the 2^c_min-key rows) fit in the tile; a phase's
    // mirror step may open a pass or follow the previous phase's last steps,
    // provided its bit is the highest in the tile.  The optimized variant
    // picks the split by a dynamic program over the step index with cost
    // kPassWeight per pass plus one per shared-memory transpose (a pass that
    // ends one step later may need a whole extra transpose); the semi variant
    // takes as many steps per pass as fit.
    std::vector<GStep> gs;
    for (int p = ksort + 1; p <= k; ++p) {
        gs.push_back({p - 1, true, p});
        for (int b = p - 2; b >= 0; --b) gs.push_back({b, false, p});
    }
    const size_t ng = gs.size();
    // Longest feasible pass from step i (every shorter run is feasible too).
    auto frontier = [&](size_t i) -> size_t {
        std::vector<int> B;
        for (int b = 0; b < c_min; ++b) B.push_back(b);
        size_t j = i;
        int nhigh = 0;
        bool flipped = false, has_low = false, has_high = false;
        while (j < ng) {
            const GStep& g = gs[j];
            const bool high = g.bit >= m;
            if (g.flip && (flipped || B.back() > g.bit)) break;
            if (!fuse && ((high && has_low) || (!high && has_high))) break;
            if (high && nhigh >= high_limit) break;
            const bool fresh = !contains(B, g.bit);
            if (fresh && (int)B.size() == m) break;
            if (fresh) {
                B.push_back(g.bit);
                std::sort(B.begin(), B.end());
            }
            flipped |= g.flip;
            has_low |= !high;
            has_high |= high;
            nhigh += high ? 1 : 0;
            ++j;
        }
        return j;
    };
    // Tile bits, local steps and descriptor of the pass over steps [i, j).
    struct PassSpec {
        std::vector<int> B;
        std::vector<LStep> ls;
        bool flipped = false;
        TileParamsBig P;
    };
    auto build_pass = [&](size_t i, size_t j, PassSpec& ps) -> bool {
        ps.B.clear();
        ps.ls.clear();
        ps.flipped = false;
        for (int b = 0; b < c_min; ++b) ps.B.push_back(b);
        for (size_t s = i; s < j; ++s) {
            if (!contains(ps.B, gs[s].bit)) ps.B.push_back(gs[s].bit);
            ps.flipped |= gs[s].flip;
        }
        // Fill the tile with the lowest free bits (longer contiguous rows).
        for (int b = 0; (int)ps.B.size() < m; ++b)
            if (!contains(ps.B, b)) ps.B.push_back(b);
        std::sort(ps.B.begin(), ps.B.end());
        for (size_t s = i; s < j; ++s) {
            const int lb = (int)(std::find(ps.B.begin(), ps.B.end(), gs[s].bit) - ps.B.begin());
            ps.ls.push_back({lb, gs[s].flip});
        }
        std::memset(&ps.P, 0, sizeof(ps.P));
        if (!map_bits(ps.P, ps.B, ps.flipped, k)) return false;
        return plan_rounds(ps.ls, cfg, vb, opt.io_direct, ps.P);
    };
    std::vector<size_t> cut;  // pass boundaries
    if (semi) {
        for (size_t i = 0; i < ng;) {
            const size_t j = frontier(i);
            if (j == i) return plan;
            cut.push_back(i);
            i = j;
        }
    } else {
        constexpr int kInf = 1 << 30;
        std::vector<int> cost(ng + 1, kInf);
        std::vector<size_t> prev(ng + 1, 0);
        cost[0] = 0;
        PassSpec ps;
        for (size_t i = 0; i < ng; ++i) {
            if (cost[i] >= kInf) continue;
            const size_t jmax = frontier(i);
            for (size_t j = i + 1; j <= jmax; ++j) {
                if (!build_pass(i, j, ps)) continue;
                const int c = cost[i] + kPassWeight + (int)ps.P.nrounds - 1;
                if (c < cost[j]) {
                    cost[j] = c;
                    prev[j] = i;
                }
            }
        }
        if (cost[ng] >= kInf) return plan;
        for (size_t j = ng; j > 0; j = prev[j]) cut.push_back(prev[j]);
        std::reverse(cut.begin(), cut.end());
    }
    for (size_t q = 0; q < cut.size(); ++q) {
        const size_t i = cut[q], j = q + 1 < cut.size() ? cut[q + 1] : ng;
        PassSpec ps;
        if (!build_pass(i, j, ps)) return plan;
        int hi = -1, lo = 64;
        for (size_t s = i; s < j; ++s) {
            hi = std::max(hi, gs[s].bit);
            lo = std::min(lo, gs[s].bit);
            if (gs[s].bit >= m) plan.global_steps += 1;
            else plan.fused_steps += 1;
        }
        bool contiguous = true;
        for (int b = 0; b < m; ++b)
            if (ps.B[b] != b) contiguous = false;
        const int kind = contiguous ? KIND_TILE_MERGE : KIND_GLOBAL;
        if (!add_pass(ps.B, ps.flipped, ps.ls, kind, gs[i].phase, hi, lo, ps.flipped)) return plan;
    }
    plan.ok = true;
    return plan;
}

}  // namespace bitonic
