// Host planner: turns a sort of n keys into a launch sequence and builds the
// tile descriptors (global mapping + register rounds) of every launch.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "desc.h"
#include "internal.h"
#include "kernel_cfg.h"

namespace bitonic {

namespace {

const TileCfg kCfgs[kNumTileCfgs] = {
#define BITONIC_CFG_ROW(ID, KT, LR, LT) {ID, (int)sizeof(KT), LR, LT},
    BITONIC_TILE_CONFIGS(BITONIC_CFG_ROW)
#undef BITONIC_CFG_ROW
};

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

// Steps at local bits top..bottom, the first one a mirror step if flip.
std::vector<LStep> merge_steps(int top, int bottom, bool flip)
{
    std::vector<LStep> s;
    for (int b = top; b >= bottom; --b) s.push_back({b, flip && b == top});
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

bool emit_round(const HostRound& hr, int log_t, int m, int vb, RoundDesc& rd)
{
    std::memset(&rd, 0, sizeof(rd));
    std::vector<int> T;
    for (int b = vb; b < m; ++b)
        if (!contains(hr.R, b)) T.push_back(b);
    if ((int)T.size() != log_t) return false;
    T = order_thread_bits(T, vb);
    for (int t = 0; t < log_t; ++t) rd.thr_loc[t] = (uint16_t)(1u << T[t]);
    for (size_t q = 0; q < hr.R.size(); ++q) {
        uint32_t v = 1u << hr.R[q];
        if (hr.R[q] == hr.mirror_bit) v |= hr.mirror;
        rd.reg_loc[q] = (uint16_t)v;
    }
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

// Lanes 0..2 on local bits vb..vb+2 that the map sends to global units:
// each quarter warp then touches one aligned 128-byte line.
bool round_coalesced(const RoundDesc& rd, const TileParams& P, int vb)
{
    for (int t = 0; t < 3; ++t) {
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

bool plan_rounds(const std::vector<LStep>& steps, const TileCfg& cfg, int vb, TileParams& P)
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
    if (rounds.empty()) {
        rounds.push_back(io_round(RR, m, vb));
    }
    std::vector<RoundDesc> out;
    for (auto& hr : rounds) {
        RoundDesc rd;
        if (!emit_round(hr, cfg.log_t, m, vb, rd)) return false;
        out.push_back(rd);
    }
    // Global loads and stores go through a coalesced layout: add a round
    // without steps (one more shared-memory transpose) where needed.
    RoundDesc io;
    if (!emit_round(io_round(RR, m, vb), cfg.log_t, m, vb, io)) return false;
    if (!round_coalesced(out.front(), P, vb)) out.insert(out.begin(), io);
    if (!round_coalesced(out.back(), P, vb)) out.push_back(io);
    if (out.size() > (size_t)kMaxRounds) return false;
    P.nrounds = (uint8_t)out.size();
    for (size_t r = 0; r < out.size(); ++r) P.rounds[r] = out[r];
    return true;
}

void map_contiguous(TileParams& P, int m, int k)
{
    P.m = (uint8_t)m;
    for (int j = 0; j < m; ++j) P.gvec[j] = 1u << j;
    int nf = 0;
    for (int b = m; b < k; ++b) P.free_bits[nf++] = (uint8_t)b;
    P.nfree = (uint8_t)nf;
    P.contiguous = 1;
}

// Tile = rows of 2^c consecutive positions at global bits lo..hi.  With flip,
// the top local bit carries the mirror step of phase p = hi + 1: it maps to
// 2^hi XOR the global bits c..lo-1 that the tile leaves out.
void map_strided(TileParams& P, int m, int c, int lo, int hi, bool flip, int k)
{
    P.m = (uint8_t)m;
    for (int j = 0; j < c; ++j) P.gvec[j] = 1u << j;
    for (int j = c; j < m; ++j) P.gvec[j] = 1u << (lo + j - c);
    if (flip) {
        uint32_t v = 1u << hi;
        for (int b = c; b < lo; ++b) v |= 1u << b;
        P.gvec[m - 1] = v;
    }
    int nf = 0;
    for (int b = c; b < lo; ++b) P.free_bits[nf++] = (uint8_t)b;
    for (int b = hi + 1; b < k; ++b) P.free_bits[nf++] = (uint8_t)b;
    P.nfree = (uint8_t)nf;
    P.contiguous = 0;
}

int choose_cfg(int key_bytes, const Options& opt)
{
    const bool semi = opt.variant == 2;
    if (key_bytes == 4) {
        if (semi) return 3;
        if (opt.tile_log2 == 13) return 1;
        return 0;
    }
    if (semi) return 6;
    if (opt.tile_log2 == 12) return 5;
    return 4;
}

}  // namespace

const TileCfg& tile_cfg(int id) { return kCfgs[id]; }

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
            for (int j = p - 1; j >= 0; --j) plan.launches.push_back({KIND_STEP, p, j, j, j == p - 1, -1, 0});
        plan.hbm_passes = (int)plan.launches.size();
        plan.global_steps = (int)plan.launches.size();
        plan.cfg = -1;
        plan.ok = true;
        return plan;
    }
    const int cfg_id = choose_cfg(key_bytes, opt);
    const TileCfg& cfg = kCfgs[cfg_id];
    const int vb = key_bytes == 4 ? 2 : 1;
    const int m = cfg.log_r + cfg.log_t;
    plan.cfg = cfg_id;
    plan.tile_log2 = m;
    const int max_gb = m - vb - 3;
    int gb = opt.global_bits > 0 ? opt.global_bits : max_gb;
    if (opt.variant == 2) gb = 1;  // semi: one stride per global pass
    gb = std::max(1, std::min(gb, max_gb));

    auto add = [&](int kind, int p, int hi, int lo, bool flip, TileParams& P, uint32_t grid) {
        plan.descs.push_back(P);
        plan.launches.push_back({kind, p, hi, lo, flip ? 1 : 0, (int)plan.descs.size() - 1, grid});
    };

    const int ksort = std::min(k, m);
    {
        TileParams P;
        std::memset(&P, 0, sizeof(P));
        map_contiguous(P, m, k);
        if (!plan_rounds(tile_sort_steps(ksort), cfg, vb, P)) return plan;
        add(KIND_TILE_SORT, ksort, ksort - 1, 0, true, P, k > m ? (1u << (k - m)) : 1u);
        plan.fused_steps += ksort * (ksort + 1) / 2;
        plan.hbm_passes += 1;
    }
    int merge_desc = -1;
    for (int p = m + 1; p <= k; ++p) {
        const int tb = p - m;
        const int npass = (tb + gb - 1) / gb;
        int hi = p - 1;
        for (int q = 0; q < npass; ++q) {
            const int cnt = tb / npass + (q < tb % npass ? 1 : 0);
            const int lo = hi - cnt + 1;
            const int c = m - cnt;
            TileParams P;
            std::memset(&P, 0, sizeof(P));
            map_strided(P, m, c, lo, hi, q == 0, k);
            if (!plan_rounds(merge_steps(m - 1, c, q == 0), cfg, vb, P)) return plan;
            add(KIND_GLOBAL, p, hi, lo, q == 0, P, 1u << (k - m));
            plan.global_steps += cnt;
            plan.hbm_passes += 1;
            hi = lo - 1;
        }
        if (merge_desc < 0) {
            TileParams P;
            std::memset(&P, 0, sizeof(P));
            map_contiguous(P, m, k);
            if (!plan_rounds(merge_steps(m - 1, 0, false), cfg, vb, P)) return plan;
            add(KIND_TILE_MERGE, p, m - 1, 0, false, P, 1u << (k - m));
            merge_desc = plan.launches.back().desc;
        } else {
            plan.launches.push_back({KIND_TILE_MERGE, p, m - 1, 0, 0, merge_desc, 1u << (k - m)});
        }
        plan.fused_steps += m;
        plan.hbm_passes += 1;
    }
    plan.ok = true;
    return plan;
}

}  // namespace bitonic
