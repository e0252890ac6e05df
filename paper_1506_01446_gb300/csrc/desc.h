// Launch descriptors shared by the host planner and the device tile engine.
//
// A tile pass works on a tile of 2^m keys.  Tile-local index L (m bits) maps
// to a global (virtual) position g0 ^ G(L), where G is linear over GF(2):
// G(L) = XOR of gvec[j] over the set bits j of L, and g0 is the CTA's base
// (its block index scattered into the global bits that are not in the tile).
// Local bits 0..c-1 map to global bits 0..c-1, so the tile is made of
// aligned rows of at least 2^c consecutive keys.
//
// The network runs on local indices in the mirror form: the first step of a
// phase pairs L with L ^ (2^(b+1) - 1) (b = the phase's top bit), the others
// pair L with L ^ 2^b, and the lower index always receives the element that
// sorts first.  A phase's first step whose span reaches global bits outside
// the tile is still a local mirror step over the whole tile: its local bit is
// the tile's top bit and maps to 2^p XOR the global bits below p that the
// tile leaves out.
//
// The steps are split into rounds.  In a round each thread holds R = 2^LOG_R
// keys in registers: register-index bits 0..VB-1 are the components of one
// 16-byte vector (local bits 0..VB-1), bits VB.. are "register bits" whose
// local vectors are reg_loc[]; thread-index bit i has local vector thr_loc[i].
// Between rounds the keys pass through shared memory (a transpose).
#pragma once

#include <stdint.h>

namespace bitonic {

constexpr int kMaxLogThreads = 10;
constexpr int kMaxRegBits = 5;        // LOG_R - VB
constexpr int kMaxRoundsSmall = 32;   // descriptors passed by value (constant bank)
constexpr int kMaxRoundsBig = 100;    // descriptors read from global memory
constexpr int kMaxStepsPerRound = 36;
constexpr int kMaxLocalBits = 16;
constexpr int kMaxCtaRuns = 4;

// Step code: register-index bit q in bits 0..3, kStepFlip set for a mirror step.
constexpr uint8_t kStepFlip = 16;

#if defined(__CUDACC__)
#define BITONIC_HD __host__ __device__
#else
#define BITONIC_HD
#endif

// Shared-memory swizzle on vector indices: the low 3 bits (the 16-byte bank
// group within a 128-byte line) are XORed with every higher 3-bit group.
// Linear over GF(2), so phys(a ^ b) = phys(a) ^ phys(b).  A quarter warp
// whose 3 lane bits sit on local vector bits of distinct residue mod 3 hits 8
// distinct bank groups.
BITONIC_HD constexpr uint32_t smem_swizzle(uint32_t lv)
{
    return lv ^ (((lv >> 3) ^ (lv >> 6) ^ (lv >> 9) ^ (lv >> 12) ^ (lv >> 15)) & 7u);
}

struct RoundDesc {
    uint16_t thr_loc[kMaxLogThreads];  // local vector of thread-index bit i
    uint16_t reg_loc[kMaxRegBits];     // local vector of register bit VB + j
    uint8_t nsteps;
    uint8_t steps[kMaxStepsPerRound];
    uint8_t pattern;                   // index into the round-pattern catalog, 0xFF = generic
    // 1 if every warp reads, in this round's layout, exactly the shared-memory
    // slots it wrote in the previous round's layout: the transpose into this
    // round then needs a warp barrier only, not a CTA barrier.
    uint8_t warp_local;
    // Byte offsets of the 16-byte shared-memory vector slots, precomputed by
    // the planner: smem_swizzle(thr_loc[i] >> VB) * 16 and
    // smem_swizzle(reg_loc[j] >> VB) * 16.  By linearity a thread's vector v
    // sits at the XOR of thr_sw over the set bits of the thread index and of
    // reg_sw over the set bits of v (tiles of at most 64 KiB: 16-bit offsets).
    uint16_t thr_sw[kMaxLogThreads];
    uint16_t reg_sw[kMaxRegBits];
};

// Global-memory side of the first (load) and last (store) rounds.
struct IoDesc {
    uint32_t thr_glob[kMaxLogThreads];  // G(thr_loc[i])
    uint32_t reg_glob[kMaxRegBits];     // G(reg_loc[j])
};

template <int MAXR>
struct TileParamsT {
    uint32_t gvec[kMaxLocalBits];     // global vector of local bit j
    IoDesc io[2];                     // [0] load round, [1] store round
    uint32_t span_mask;               // OR of gvec: the tile's positions lie in
                                      // [g0 & ~span_mask, g0 | span_mask]
    uint8_t run_shift[kMaxCtaRuns];   // CTA index bits go to global bits
    uint8_t run_width[kMaxCtaRuns];   //   run_shift[r] .. run_shift[r]+run_width[r]-1
    uint8_t m;                        // local bits
    uint8_t nruns;
    uint8_t contiguous;               // tile is one aligned block of 2^m positions
    uint8_t nrounds;
    uint8_t row_log;                  // tile rows: 2^row_log consecutive positions (local bits below
                                      // row_log map to the same global bits)
    uint8_t pad_[3];
    RoundDesc rounds[MAXR];
};

using TileParams = TileParamsT<kMaxRoundsSmall>;
using TileParamsBig = TileParamsT<kMaxRoundsBig>;

}  // namespace bitonic
