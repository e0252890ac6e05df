// Device side of the tile engine: the register network (Section 4.2), the
// shared-memory transposes between rounds (Section 4.1) and the global
// loads / stores with virtual padding.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "desc.h"

namespace bitonic {

template <typename K>
struct KeyTraits;

template <>
struct KeyTraits<uint32_t> {
    static constexpr int VEC = 4;  // keys per 16-byte vector
    static constexpr int VB = 2;   // log2(VEC)
    using Vec = uint4;
    static constexpr uint32_t kMax = 0xFFFFFFFFu;
};

template <>
struct KeyTraits<uint64_t> {
    static constexpr int VEC = 2;
    static constexpr int VB = 1;
    using Vec = ulonglong2;
    static constexpr uint64_t kMax = 0xFFFFFFFFFFFFFFFFull;
};


// Multipliers 1 and 2^32 - 1 for the multiply-add form of a 4-byte
// compare-exchange.  Read from constant memory, so the compiler cannot turn
// the multiply-adds back into integer-ALU adds.
static __constant__ uint32_t c_ce_mul[2] = {1u, 0xFFFFFFFFu};

// Of every three 4-byte compare-exchanges of a step, how many take the
// larger key as a + b - min(a, b) with two multiply-adds (FMA pipe) instead
// of a max (integer ALU).  A compare-exchange is otherwise two min/max on
// the integer ALU while the FMA pipe idles.
#ifndef BITONIC_CE_FMA_THIRDS
#define BITONIC_CE_FMA_THIRDS 2
#endif

// Of every three 8-byte compare-exchanges, how many take each 32-bit half
// of the larger key as a + b - min(a, b) with two multiply-adds (the
// halves are independent: the minimum is one of the two keys, so each half
// of it is that key's half).  The others use a ^ b ^ min(a, b).  With all
// three, the compare and the selects of the minimum (integer ALU) and the
// four multiply-adds (FMA pipe) split a compare-exchange evenly between the
// two pipes: 6.81 ms against 7.13 ms (none) and 6.86 ms (two of three) for
// 2^26 uint64 keys.
#ifndef BITONIC_CE64_FMA_THIRDS
#define BITONIC_CE64_FMA_THIRDS 3
#endif

// Compare-exchange: the lower register receives the key that sorts first.
// third: the compare-exchange's position modulo 3 within its step, which
// picks its form (constant once the caller's loop unrolls).  4-byte keys:
// the multiply-add form (exact modulo 2^32, since the minimum is one of the
// two keys) or a min and a max.  8-byte keys: one 64-bit compare and two
// selects for the minimum, then the larger key from multiply-adds or from
// logic ops (the latter 9.0 vs 6.9 compare-exchanges per clock per SM
// against two more selects in a register-only probe).
template <bool DESC, typename K>
__device__ __forceinline__ void cmpx(K& a, K& b, int third = 3)
{
    K lo, hi;
    if (sizeof(K) == 4 && third < BITONIC_CE_FMA_THIRDS) {
        lo = a < b ? a : b;
        const K sum = a * c_ce_mul[0] + b;
        hi = lo * c_ce_mul[1] + sum;
    } else if (sizeof(K) == 8 && third < BITONIC_CE64_FMA_THIRDS) {
        lo = a < b ? a : b;
        const uint32_t s0 = (uint32_t)a * c_ce_mul[0] + (uint32_t)b;
        const uint32_t s1 = (uint32_t)(a >> 32) * c_ce_mul[0] + (uint32_t)(b >> 32);
        const uint32_t h0 = (uint32_t)lo * c_ce_mul[1] + s0;
        const uint32_t h1 = (uint32_t)(lo >> 32) * c_ce_mul[1] + s1;
        hi = ((K)h1 << 32) | h0;
    } else if (sizeof(K) == 8) {
        lo = a < b ? a : b;
        hi = a ^ b ^ lo;
    } else {
        lo = a < b ? a : b;
        hi = a < b ? b : a;
    }
    a = DESC ? hi : lo;
    b = DESC ? lo : hi;
}

// One network step on the register array.  FLIP: mirror step at register bit
// Q (pairs i with i ^ (2^(Q+1) - 1)); otherwise half-cleaner (i with i ^ 2^Q).
template <int Q, bool FLIP, bool DESC, typename K, int R>
__device__ __forceinline__ void net_step(K (&r)[R])
{
#pragma unroll
    for (int i = 0; i < R; ++i) {
        if (i & (1 << Q)) continue;
        const int j = FLIP ? (i ^ ((2 << Q) - 1)) : (i | (1 << Q));
        cmpx<DESC>(r[i], r[j], (i + Q) % 3);
    }
}

template <bool DESC, typename K, int R>
__device__ __forceinline__ void run_step(K (&r)[R], int code)
{
    constexpr int LOG_R = (R >= 128) ? 7 : (R >= 64) ? 6 : (R >= 32) ? 5 : (R >= 16) ? 4 : (R >= 8) ? 3 : (R >= 4) ? 2 : 1;
#define BITONIC_STEP_CASE(Q)                                                  \
    case Q:                                                                   \
        if constexpr (Q < LOG_R) net_step<Q, false, DESC>(r);                 \
        break;                                                                \
    case Q + kStepFlip:                                                       \
        if constexpr (Q < LOG_R) net_step<Q, true, DESC>(r);                  \
        break;
    switch (code) {
        BITONIC_STEP_CASE(0)
        BITONIC_STEP_CASE(1)
        BITONIC_STEP_CASE(2)
        BITONIC_STEP_CASE(3)
        BITONIC_STEP_CASE(4)
        BITONIC_STEP_CASE(5)
        BITONIC_STEP_CASE(6)
        default: break;
    }
#undef BITONIC_STEP_CASE
}

template <bool DESC, typename K, int R>
__device__ __forceinline__ void run_round_steps(K (&r)[R], const RoundDesc& rd)
{
    const int ns = rd.nsteps;
    for (int s = 0; s < ns; ++s) run_step<DESC>(r, (int)rd.steps[s]);
}

// Thread part of a round's local index: XOR of thr_loc[i] over set bits i of x.
template <int LOG_T>
__device__ __forceinline__ uint32_t thread_local_index(const RoundDesc& rd, uint32_t x)
{
    uint32_t L = 0;
#pragma unroll
    for (int i = 0; i < LOG_T; ++i)
        if ((x >> i) & 1u) L ^= rd.thr_loc[i];
    return L;
}

// Thread part of a round's shared-memory slot (a byte offset): XOR of
// thr_sw[i] over set bits i of x.
template <int LOG_T>
__device__ __forceinline__ uint32_t thread_smem_slot(const RoundDesc& rd, uint32_t x)
{
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < LOG_T; ++i)
        if ((x >> i) & 1u) s ^= rd.thr_sw[i];
    return s;
}

// Register part of vector v's local index (v indexes the R / VEC vectors).
template <int NREG>
__device__ __forceinline__ uint32_t reg_local_index(const uint32_t (&rv)[NREG], int v)
{
    uint32_t L = 0;
#pragma unroll
    for (int j = 0; j < NREG; ++j)
        if ((v >> j) & 1) L ^= rv[j];
    return L;
}

// CTA base position: the bits of the CTA index scattered into the runs of
// global bits that the tile does not cover.
template <class PT>
__device__ __forceinline__ uint32_t cta_base(const PT& P, uint32_t cta)
{
    uint32_t g = 0;
    const int nr = P.nruns;
#pragma unroll
    for (int r = 0; r < kMaxCtaRuns; ++r) {
        if (r < nr) {
            const uint32_t w = P.run_width[r];
            g |= (cta & ((1u << w) - 1u)) << P.run_shift[r];
            cta >>= w;
        }
    }
    return g;
}

// Global position of this thread's part of an I/O round's layout.
template <int LOG_T>
__device__ __forceinline__ uint32_t io_thread_global(const IoDesc& io, uint32_t x)
{
    uint32_t g = 0;
#pragma unroll
    for (int i = 0; i < LOG_T; ++i)
        if ((x >> i) & 1u) g ^= io.thr_glob[i];
    return g;
}

// 16-byte global load; CG: cached in L2 only (ld.global.cg), for data that
// other CTAs of the same launch wrote (the L1 of this SM may hold an older
// copy of the line).
template <bool CG, typename V>
__device__ __forceinline__ V load_vec(const V* p)
{
    if constexpr (CG)
        return __ldcg(p);
    else
        return *p;
}

template <bool CG, typename K>
__device__ __forceinline__ K load_key(const K* p)
{
    if constexpr (CG)
        return __ldcg(p);
    else
        return *p;
}

template <typename K>
__device__ __forceinline__ void vec_to_regs(const typename KeyTraits<K>::Vec& w, K* r);

template <>
__device__ __forceinline__ void vec_to_regs<uint32_t>(const uint4& w, uint32_t* r)
{
    r[0] = w.x; r[1] = w.y; r[2] = w.z; r[3] = w.w;
}

template <>
__device__ __forceinline__ void vec_to_regs<uint64_t>(const ulonglong2& w, uint64_t* r)
{
    r[0] = w.x; r[1] = w.y;
}

template <typename K>
__device__ __forceinline__ typename KeyTraits<K>::Vec regs_to_vec(const K* r);

template <>
__device__ __forceinline__ uint4 regs_to_vec<uint32_t>(const uint32_t* r)
{
    return make_uint4(r[0], r[1], r[2], r[3]);
}

template <>
__device__ __forceinline__ ulonglong2 regs_to_vec<uint64_t>(const uint64_t* r)
{
    return make_ulonglong2(r[0], r[1]);
}

// Order-preserving key map, applied to real keys on a sort's first load and
// last store: v -> v ^ (fill(v ^ s) & a) ^ b, fill(x) = all ones if x's top
// bit is set, else zero.  With a = 0 it is the XOR with b (b = ~0: the
// complement that turns a descending sort into an ascending one; b = the
// sign bit: signed integers).  Floats use a = ~sign bit, which flips the
// magnitude bits of negative keys (IEEE 754 totalOrder becomes unsigned
// order); the inverse map on the store takes s = ~0.
template <typename K>
struct KeyMap {
    K a, b, s;
    __device__ __forceinline__ K operator()(K v) const
    {
        using S = typename std::make_signed<K>::type;
        const K fill = (K)((S)(v ^ s) >> (8 * sizeof(K) - 1));
        return v ^ (fill & a) ^ b;
    }
};

// The tile engine for one CTA.  LOG_R keys-per-thread bits, LOG_T thread bits.
template <typename K, bool DESC, int LOG_R, int LOG_T>
struct Tile {
    static constexpr int R = 1 << LOG_R;
    static constexpr int VEC = KeyTraits<K>::VEC;
    static constexpr int VB = KeyTraits<K>::VB;
    static constexpr int NV = R / VEC;           // vectors per thread
    static constexpr int NREG = LOG_R - VB;      // register bits beyond the vector
    using Vec = typename KeyTraits<K>::Vec;
    static_assert(NREG >= 1 && NREG <= kMaxRegBits, "register bits out of range");
    static_assert(LOG_T <= kMaxLogThreads, "too many threads");

    static constexpr K kFrontPad = DESC ? KeyTraits<K>::kMax : K(0);
    static constexpr K kTailPad = DESC ? K(0) : KeyTraits<K>::kMax;

    K r[R];

    __device__ __forceinline__ void load_reg_vectors(const RoundDesc& rd, uint32_t (&rv)[NREG])
    {
#pragma unroll
        for (int j = 0; j < NREG; ++j) rv[j] = rd.reg_loc[j];
    }

    // Global load in the load round's layout.  base points at virtual
    // position 0; positions [lo, hi) hold real keys, others are pads.
    template <bool CG = false>
    __device__ __forceinline__ void load_global(const K* __restrict__ base, uint32_t lo, uint32_t hi,
                                                const IoDesc& io, uint32_t g0, uint32_t x, KeyMap<K> m)
    {
        const uint32_t gt = g0 ^ io_thread_global<LOG_T>(io, x);
        uint32_t gr[NREG];
#pragma unroll
        for (int j = 0; j < NREG; ++j) gr[j] = io.reg_glob[j];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const uint32_t pos = gt ^ reg_local_index<NREG>(gr, v);
            K* dst = r + v * VEC;
            if (pos >= lo && pos + VEC <= hi) {
                vec_to_regs<K>(load_vec<CG>(reinterpret_cast<const Vec*>(base + pos)), dst);
#pragma unroll
                for (int c = 0; c < VEC; ++c) dst[c] = m(dst[c]);
            } else {
#pragma unroll
                for (int c = 0; c < VEC; ++c) {
                    const uint32_t p = pos + c;
                    dst[c] = p < lo ? kFrontPad : (p >= hi ? kTailPad : m(load_key<CG>(base + p)));
                }
            }
        }
    }

    __device__ __forceinline__ void store_global(K* __restrict__ base, uint32_t lo, uint32_t hi,
                                                 const IoDesc& io, uint32_t g0, uint32_t x, KeyMap<K> m)
    {
        const uint32_t gt = g0 ^ io_thread_global<LOG_T>(io, x);
        uint32_t gr[NREG];
#pragma unroll
        for (int j = 0; j < NREG; ++j) gr[j] = io.reg_glob[j];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const uint32_t pos = gt ^ reg_local_index<NREG>(gr, v);
            K src[VEC];
#pragma unroll
            for (int c = 0; c < VEC; ++c) src[c] = m(r[v * VEC + c]);
            if (pos >= lo && pos + VEC <= hi) {
                *reinterpret_cast<Vec*>(base + pos) = regs_to_vec<K>(src);
            } else if (pos + VEC > lo && pos < hi) {
#pragma unroll
                for (int c = 0; c < VEC; ++c) {
                    const uint32_t p = pos + c;
                    if (p >= lo && p < hi) base[p] = src[c];
                }
            }
        }
    }

    // Shared-memory addresses (in vectors) of this thread's vectors under rd.
    __device__ __forceinline__ void smem_write(Vec* sm, const RoundDesc& rd, uint32_t x)
    {
        uint32_t pr[NREG];
#pragma unroll
        for (int j = 0; j < NREG; ++j) pr[j] = rd.reg_sw[j];
        const uint32_t pt = thread_smem_slot<LOG_T>(rd, x);
        unsigned char* sb = reinterpret_cast<unsigned char*>(sm);
#pragma unroll
        for (int v = 0; v < NV; ++v)
            *reinterpret_cast<Vec*>(sb + (pt ^ reg_local_index<NREG>(pr, v))) = regs_to_vec<K>(r + v * VEC);
    }

    // Global load / store for tiles that lie wholly inside [lo, hi).
    template <bool CG = false>
    __device__ __forceinline__ void load_global_interior(const K* __restrict__ base, const IoDesc& io, uint32_t g0,
                                                         uint32_t x, KeyMap<K> m)
    {
        const uint32_t gt = g0 ^ io_thread_global<LOG_T>(io, x);
        uint32_t gr[NREG];
#pragma unroll
        for (int j = 0; j < NREG; ++j) gr[j] = io.reg_glob[j];
#pragma unroll
        for (int v = 0; v < NV; ++v)
            vec_to_regs<K>(load_vec<CG>(reinterpret_cast<const Vec*>(base + (gt ^ reg_local_index<NREG>(gr, v)))),
                           r + v * VEC);
        apply_map(m);
    }

    // Applies m to every register: nothing for the identity, one XOR per key
    // when a = 0 (branches are uniform across the CTA).
    __device__ __forceinline__ void apply_map(KeyMap<K> m)
    {
        if (m.a) {
#pragma unroll
            for (int i = 0; i < R; ++i) r[i] = m(r[i]);
        } else if (m.b) {
#pragma unroll
            for (int i = 0; i < R; ++i) r[i] ^= m.b;
        }
    }

    __device__ __forceinline__ void store_global_interior(K* __restrict__ base, const IoDesc& io, uint32_t g0,
                                                          uint32_t x, KeyMap<K> m)
    {
        apply_map(m);
        const uint32_t gt = g0 ^ io_thread_global<LOG_T>(io, x);
        uint32_t gr[NREG];
#pragma unroll
        for (int j = 0; j < NREG; ++j) gr[j] = io.reg_glob[j];
#pragma unroll
        for (int v = 0; v < NV; ++v)
            *reinterpret_cast<Vec*>(base + (gt ^ reg_local_index<NREG>(gr, v))) = regs_to_vec<K>(r + v * VEC);
    }

    // Read of a tile stored linearly by local index (as the bulk copies land),
    // complementing every key by cm.
    __device__ __forceinline__ void smem_read_linear(const Vec* sm, const RoundDesc& rd, uint32_t x, K cm)
    {
        uint32_t rv[NREG];
        load_reg_vectors(rd, rv);
        uint32_t pr[NREG];
#pragma unroll
        for (int j = 0; j < NREG; ++j) pr[j] = rv[j] >> VB;
        const uint32_t pt = thread_local_index<LOG_T>(rd, x) >> VB;
#pragma unroll
        for (int v = 0; v < NV; ++v) vec_to_regs<K>(sm[pt ^ reg_local_index<NREG>(pr, v)], r + v * VEC);
        if (cm) {
#pragma unroll
            for (int i = 0; i < R; ++i) r[i] ^= cm;
        }
    }

    __device__ __forceinline__ void smem_read(const Vec* sm, const RoundDesc& rd, uint32_t x)
    {
        uint32_t pr[NREG];
#pragma unroll
        for (int j = 0; j < NREG; ++j) pr[j] = rd.reg_sw[j];
        const uint32_t pt = thread_smem_slot<LOG_T>(rd, x);
        const unsigned char* sb = reinterpret_cast<const unsigned char*>(sm);
#pragma unroll
        for (int v = 0; v < NV; ++v)
            vec_to_regs<K>(*reinterpret_cast<const Vec*>(sb + (pt ^ reg_local_index<NREG>(pr, v))), r + v * VEC);
    }
};

}  // namespace bitonic
