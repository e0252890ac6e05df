/*
 * CPU oracle for the bitonic sorting library -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct C.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library; the GPU
 * library shares no code, header, table or helper with it.
 *
 * What it computes (all results are unique, so no tolerance applies):
 *   keys     the non-decreasing (or non-increasing) permutation of the input;
 *   pairs    the permutation ordered by (key, original index), ties by
 *            ascending index in both directions, values travelling with keys;
 *   segments each segment [off[i], off[i+1]) sorted ascending on its own.
 *
 * Two independent routes:
 *   1. the bitonic sorting network exactly as Section 3.1 states it: k phases
 *      for n = 2^k, phase r merging 2^(k-r) subsequences of length 2^r in
 *      alternating directions, each merge taking r half-cleaner steps of n/2
 *      compare-exchanges (counted, Section 3.2's closed forms);
 *   2. a top-down stable merge sort that shares no code with route 1.
 * A median-of-three Hoare quicksort (the CPU comparison of Section 5,
 * Table 1) is included as a timed baseline.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - block b of phase r < k is ascending iff b is even (Section 3.1 says
 *     only that directions alternate; the flag first_descending runs the
 *     other order, which must give the same output);
 *   - n that is not a power of two is padded to N = next_pow2(n) with
 *     0xFFFFFFFF keys (pairs: key 0xFFFFFFFF and index n..N-1);
 *   - descending keys-only flips every block's direction, so the pads end up
 *     first and the result is the last n positions; descending pairs sort
 *     (~key, index) ascending;
 *   - other key types (int32, float32, uint64, int64, float64) use the same
 *     network with the type's own order: signed integers numerically, floats
 *     by IEEE 754-2008 totalOrder (clause 5.10: -NaN < -inf < ... < -0 < +0
 *     < ... < +inf < +NaN, NaNs ordered by payload), which fixes where
 *     signed zeros and NaNs go; pads are the type's last key.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0   /* > 0 only in test builds that plant a mistake */
#endif

typedef struct {
    uint64_t compare_exchanges;
    uint64_t steps;
    uint64_t phases;
} oracle_counts;

#define ORACLE_OK 0
#define ORACLE_ERR_INVALID 1
#define ORACLE_ERR_NOMEM 3

static uint64_t next_pow2_u64(uint64_t n)
{
    uint64_t N = 1;
    while (N < n) N <<= 1;
    return N;
}

static int log2_u64(uint64_t N)
{
    int k = 0;
    while (((uint64_t)1 << k) < N) ++k;
    return k;
}

/* ------------------------------------------------------------------------ */
/* Route 1: the bitonic sorting network of Section 3.1.                       */
/* ------------------------------------------------------------------------ */

/* Direction of block containing index i in phase p (1-based) of a k-phase
 * network: returns 1 for ascending.  The last phase has a single block in the
 * requested direction. */
static int block_ascending(uint64_t i, int p, int k, int ascending, int first_descending)
{
    if (p == k) return ascending;
#if ORACLE_MUTANT == 2
    int odd = (int)((i >> (p - 1)) & 1);   /* planted: wrong block index bit */
#else
    int odd = (int)((i >> p) & 1);          /* block number = i / 2^p */
#endif
    int up = first_descending ? odd : !odd;
    return ascending ? up : !up;            /* descending flips every block */
}

/* Sort a[0..N) (N = 2^k) with the network; counts every compare-exchange. */
static void network_u32(uint32_t *a, uint64_t N, int ascending, int first_descending,
                        oracle_counts *c)
{
    int k = log2_u64(N);
    for (int p = 1; p <= k; ++p) {                    /* phase p: blocks of 2^p */
        c->phases += 1;
#if ORACLE_MUTANT == 4
        for (int j = p; j >= 1; --j) {                /* planted: strides shifted */
#elif ORACLE_MUTANT == 1
        for (int j = p - 1; j >= 1; --j) {            /* planted: last step dropped */
#else
        for (int j = p - 1; j >= 0; --j) {            /* p steps, stride 2^j */
#endif
            uint64_t d = (uint64_t)1 << j;
            c->steps += 1;
            for (uint64_t i = 0; i < N; ++i) {
                if (i & d) continue;                  /* i is the lower element */
                uint64_t partner = i | d;
                if (partner >= N) continue;
                int up = block_ascending(i, p, k, ascending, first_descending);
#if ORACLE_MUTANT == 3
                int out_of_order = up ? (a[i] < a[partner]) : (a[i] > a[partner]);
#else
                int out_of_order = up ? (a[i] > a[partner]) : (a[i] < a[partner]);
#endif
                if (out_of_order) {
                    uint32_t t = a[i];
                    a[i] = a[partner];
                    a[partner] = t;
                }
                c->compare_exchanges += 1;
            }
        }
    }
}

int oracle_bitonic_sort_u32(uint32_t *keys, uint64_t n, int ascending, int first_descending,
                            oracle_counts *counts)
{
    oracle_counts local = {0, 0, 0};
    if (!counts) counts = &local;
    memset(counts, 0, sizeof(*counts));
    if (n == 0) return ORACLE_OK;
    if (!keys) return ORACLE_ERR_INVALID;
    uint64_t N = next_pow2_u64(n);
    uint32_t *a = (uint32_t *)malloc(N * sizeof(uint32_t));
    if (!a) return ORACLE_ERR_NOMEM;
    memcpy(a, keys, n * sizeof(uint32_t));
    for (uint64_t i = n; i < N; ++i) a[i] = 0xFFFFFFFFu;
    network_u32(a, N, ascending, first_descending, counts);
    /* ascending: pads (maximal) end last; descending: they end first. */
    memcpy(keys, ascending ? a : a + (N - n), n * sizeof(uint32_t));
    free(a);
    return ORACLE_OK;
}

/* Bitonic merge of a bitonic sequence a[0..n), n = 2^r: the r half-cleaner
 * steps of Section 3.1 (stride n/2 first), stopping after max_steps steps if
 * max_steps >= 0. */
int oracle_bitonic_merge_u32(uint32_t *a, uint64_t n, int ascending, int max_steps)
{
    if (n == 0) return ORACLE_OK;
    if (!a || next_pow2_u64(n) != n) return ORACLE_ERR_INVALID;
    int r = log2_u64(n), done = 0;
    for (int j = r - 1; j >= 0; --j) {
        if (max_steps >= 0 && done >= max_steps) break;
        uint64_t d = (uint64_t)1 << j;
        for (uint64_t i = 0; i < n; ++i) {
            if (i & d) continue;
            int out_of_order = ascending ? (a[i] > a[i | d]) : (a[i] < a[i | d]);
            if (out_of_order) { uint32_t t = a[i]; a[i] = a[i | d]; a[i | d] = t; }
        }
        ++done;
    }
    return ORACLE_OK;
}

typedef struct { uint32_t key; uint32_t idx; } kv_elem;

static int kv_greater(kv_elem x, kv_elem y)
{
    if (x.key != y.key) return x.key > y.key;
#if ORACLE_MUTANT == 6
    return x.idx < y.idx;                    /* planted: tie order reversed */
#else
    return x.idx > y.idx;
#endif
}

int oracle_bitonic_sort_pairs_u32(uint32_t *keys, uint32_t *vals, uint64_t n, int ascending,
                                  oracle_counts *counts)
{
    oracle_counts local = {0, 0, 0};
    if (!counts) counts = &local;
    memset(counts, 0, sizeof(*counts));
    if (n == 0) return ORACLE_OK;
    if (!keys || !vals || n > 0xFFFFFFFFull) return ORACLE_ERR_INVALID;
    uint64_t N = next_pow2_u64(n);
    kv_elem *a = (kv_elem *)malloc(N * sizeof(kv_elem));
    uint32_t *v = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!a || !v) { free(a); free(v); return ORACLE_ERR_NOMEM; }
    memcpy(v, vals, n * sizeof(uint32_t));
    for (uint64_t i = 0; i < N; ++i) {
        a[i].key = i < n ? (ascending ? keys[i] : ~keys[i]) : 0xFFFFFFFFu;
        a[i].idx = (uint32_t)i;
    }
    int k = log2_u64(N);
    for (int p = 1; p <= k; ++p) {
        counts->phases += 1;
        for (int j = p - 1; j >= 0; --j) {
            uint64_t d = (uint64_t)1 << j;
            counts->steps += 1;
            for (uint64_t i = 0; i < N; ++i) {
                if (i & d) continue;
                int up = block_ascending(i, p, k, 1, 0);
                int out_of_order = up ? kv_greater(a[i], a[i | d]) : kv_greater(a[i | d], a[i]);
                if (out_of_order) { kv_elem t = a[i]; a[i] = a[i | d]; a[i | d] = t; }
                counts->compare_exchanges += 1;
            }
        }
    }
    for (uint64_t i = 0; i < n; ++i) {
        keys[i] = ascending ? a[i].key : ~a[i].key;
        vals[i] = v[a[i].idx];
    }
    free(a);
    free(v);
    return ORACLE_OK;
}

/* Each segment [offsets[s], offsets[s+1]) sorted ascending by the network. */
int oracle_segmented_sort_u32(uint32_t *keys, const int32_t *offsets, int64_t nseg)
{
    if (nseg < 0 || (nseg > 0 && (!keys || !offsets))) return ORACLE_ERR_INVALID;
    for (int64_t s = 0; s < nseg; ++s) {
        if (offsets[s + 1] < offsets[s]) return ORACLE_ERR_INVALID;
        int rc = oracle_bitonic_sort_u32(keys + offsets[s], (uint64_t)(offsets[s + 1] - offsets[s]),
                                         1, 0, NULL);
        if (rc) return rc;
    }
    return ORACLE_OK;
}

int oracle_segmented_sort_pairs_u32(uint32_t *keys, uint32_t *vals, const int32_t *offsets,
                                    int64_t nseg)
{
    if (nseg < 0 || (nseg > 0 && (!keys || !vals || !offsets))) return ORACLE_ERR_INVALID;
    for (int64_t s = 0; s < nseg; ++s) {
        if (offsets[s + 1] < offsets[s]) return ORACLE_ERR_INVALID;
        int rc = oracle_bitonic_sort_pairs_u32(keys + offsets[s], vals + offsets[s],
                                               (uint64_t)(offsets[s + 1] - offsets[s]), 1, NULL);
        if (rc) return rc;
    }
    return ORACLE_OK;
}

/* 0-1 principle (Knuth, TAOCP vol. 3, 5.3.4): a comparator network sorts
 * every input iff it sorts every 0/1 input.  Runs the network on all 2^m
 * zero-one inputs of length m and returns how many come out wrong (unsorted
 * or with a changed number of ones). */
uint64_t oracle_zero_one_failures(int m, int ascending, int first_descending)
{
    if (m < 0 || m > 24) return (uint64_t)-1;
    uint64_t failures = 0, total = (uint64_t)1 << m;
    uint32_t *a = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    if (!a) return (uint64_t)-1;
    for (uint64_t mask = 0; mask < total; ++mask) {
        int ones = 0;
        for (int i = 0; i < m; ++i) { a[i] = (uint32_t)((mask >> i) & 1); ones += (int)a[i]; }
        oracle_bitonic_sort_u32(a, (uint64_t)m, ascending, first_descending, NULL);
        int bad = 0, ones_after = 0;
        for (int i = 0; i < m; ++i) {
            ones_after += (int)a[i];
            if (i && (ascending ? a[i - 1] > a[i] : a[i - 1] < a[i])) bad = 1;
        }
        if (bad || ones != ones_after) ++failures;
    }
    free(a);
    return failures;
}

/* ------------------------------------------------------------------------ */
/* Route 2: top-down stable merge sort (independent of route 1).             */
/* ------------------------------------------------------------------------ */

static int before_u32(uint32_t x, uint32_t y, int ascending)
{
    return ascending ? x < y : x > y;
}

static void merge_rec_u32(uint32_t *a, uint32_t *tmp, uint64_t lo, uint64_t hi, int ascending)
{
    if (hi - lo < 2) return;
    uint64_t mid = lo + (hi - lo) / 2;
    merge_rec_u32(a, tmp, lo, mid, ascending);
    merge_rec_u32(a, tmp, mid, hi, ascending);
    uint64_t i = lo, j = mid, o = lo;
    while (i < mid && j < hi) {
        /* take from the right run only if strictly before: keeps it stable */
        if (before_u32(a[j], a[i], ascending)) tmp[o++] = a[j++];
        else tmp[o++] = a[i++];
    }
    while (i < mid) tmp[o++] = a[i++];
    while (j < hi) tmp[o++] = a[j++];
    memcpy(a + lo, tmp + lo, (hi - lo) * sizeof(uint32_t));
}

int oracle_merge_sort_u32(uint32_t *keys, uint64_t n, int ascending)
{
    if (n < 2) return ORACLE_OK;
    if (!keys) return ORACLE_ERR_INVALID;
    uint32_t *tmp = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!tmp) return ORACLE_ERR_NOMEM;
    merge_rec_u32(keys, tmp, 0, n, ascending);
    free(tmp);
    return ORACLE_OK;
}

static void merge_rec_pairs(uint32_t *k, uint32_t *v, uint32_t *tk, uint32_t *tv, uint64_t lo,
                            uint64_t hi, int ascending)
{
    if (hi - lo < 2) return;
    uint64_t mid = lo + (hi - lo) / 2;
    merge_rec_pairs(k, v, tk, tv, lo, mid, ascending);
    merge_rec_pairs(k, v, tk, tv, mid, hi, ascending);
    uint64_t i = lo, j = mid, o = lo;
    while (i < mid && j < hi) {
#if ORACLE_MUTANT == 5
        int take_right = !before_u32(k[i], k[j], ascending);   /* planted: unstable */
#else
        int take_right = before_u32(k[j], k[i], ascending);
#endif
        if (take_right) { tk[o] = k[j]; tv[o++] = v[j++]; }
        else { tk[o] = k[i]; tv[o++] = v[i++]; }
    }
    while (i < mid) { tk[o] = k[i]; tv[o++] = v[i++]; }
    while (j < hi) { tk[o] = k[j]; tv[o++] = v[j++]; }
    memcpy(k + lo, tk + lo, (hi - lo) * sizeof(uint32_t));
    memcpy(v + lo, tv + lo, (hi - lo) * sizeof(uint32_t));
}

/* Stable: equal keys keep their input order, i.e. ascending original index,
 * in both directions. */
int oracle_merge_sort_pairs_u32(uint32_t *keys, uint32_t *vals, uint64_t n, int ascending)
{
    if (n < 2) return ORACLE_OK;
    if (!keys || !vals) return ORACLE_ERR_INVALID;
    uint32_t *tk = (uint32_t *)malloc(n * sizeof(uint32_t));
    uint32_t *tv = (uint32_t *)malloc(n * sizeof(uint32_t));
    if (!tk || !tv) { free(tk); free(tv); return ORACLE_ERR_NOMEM; }
    merge_rec_pairs(keys, vals, tk, tv, 0, n, ascending);
    free(tk);
    free(tv);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* CPU comparison sort of Section 5: median-of-three Hoare quicksort.        */
/* ------------------------------------------------------------------------ */

static void insertion_u32(uint32_t *a, int64_t lo, int64_t hi)
{
    for (int64_t i = lo + 1; i <= hi; ++i) {
        uint32_t x = a[i];
        int64_t j = i - 1;
        while (j >= lo && a[j] > x) { a[j + 1] = a[j]; --j; }
        a[j + 1] = x;
    }
}

static void quick_rec_u32(uint32_t *a, int64_t lo, int64_t hi)
{
    while (hi - lo > 16) {
        int64_t mid = lo + (hi - lo) / 2;
        uint32_t x = a[lo], y = a[mid], z = a[hi];
        uint32_t pivot = (x < y) ? ((y < z) ? y : (x < z ? z : x)) : ((x < z) ? x : (y < z ? z : y));
        int64_t i = lo - 1, j = hi + 1;
        for (;;) {
            do { ++i; } while (a[i] < pivot);
            do { --j; } while (a[j] > pivot);
            if (i >= j) break;
            uint32_t t = a[i]; a[i] = a[j]; a[j] = t;
        }
        /* recurse into the smaller side, loop on the larger */
        if (j - lo < hi - j) { quick_rec_u32(a, lo, j); lo = j + 1; }
        else { quick_rec_u32(a, j + 1, hi); hi = j; }
    }
    insertion_u32(a, lo, hi);
}

void oracle_quicksort_u32(uint32_t *keys, uint64_t n)
{
    if (n < 2 || !keys) return;
    quick_rec_u32(keys, 0, (int64_t)n - 1);
}

/* ------------------------------------------------------------------------ */
/* Checkers.                                                                  */
/* ------------------------------------------------------------------------ */

int oracle_is_sorted_u32(const uint32_t *a, uint64_t n, int ascending)
{
    for (uint64_t i = 1; i < n; ++i)
        if (ascending ? a[i - 1] > a[i] : a[i - 1] < a[i]) return 0;
    return 1;
}

/* Multiset equality by an open-addressing histogram: +1 per key of a, -1 per
 * key of b; equal iff every count ends at zero.  Returns 1/0, or -1 when out
 * of memory. */
int oracle_same_multiset_u32(const uint32_t *a, const uint32_t *b, uint64_t n)
{
    if (n == 0) return 1;
    uint64_t cap = next_pow2_u64(2 * n);
    uint32_t *slot_key = (uint32_t *)malloc(cap * sizeof(uint32_t));
    int64_t *slot_cnt = (int64_t *)calloc(cap, sizeof(int64_t));
    uint8_t *used = (uint8_t *)calloc(cap, 1);
    if (!slot_key || !slot_cnt || !used) { free(slot_key); free(slot_cnt); free(used); return -1; }
    for (int pass = 0; pass < 2; ++pass) {
        const uint32_t *src = pass ? b : a;
        int64_t delta = pass ? -1 : 1;
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t h = ((uint64_t)src[i] * 0x9E3779B97F4A7C15ull) >> 17;
            for (;;) {
                uint64_t s = h & (cap - 1);
                if (!used[s]) { used[s] = 1; slot_key[s] = src[i]; slot_cnt[s] = delta; break; }
                if (slot_key[s] == src[i]) { slot_cnt[s] += delta; break; }
                ++h;
            }
        }
    }
    int same = 1;
    for (uint64_t s = 0; s < cap; ++s)
        if (used[s] && slot_cnt[s] != 0) { same = 0; break; }
    free(slot_key);
    free(slot_cnt);
    free(used);
    return same;
}

/* ------------------------------------------------------------------------ */
/* Other key types: the same Section 3.1 network, with each type's order     */
/* written out from its definition (no bit tricks).                           */
/* ------------------------------------------------------------------------ */

#define ORACLE_KEY_I32 1
#define ORACLE_KEY_F32 2
#define ORACLE_KEY_U64 3
#define ORACLE_KEY_I64 4
#define ORACLE_KEY_F64 5

/* IEEE 754-2008 totalOrder (clause 5.10) as a strict "x before y":
 *   - a key with the sign bit set comes before one without it (so -0 before
 *     +0, and a negative NaN before everything, a positive NaN after);
 *   - same sign, neither a NaN: the numeric order (equal zeros tie);
 *   - same sign, NaNs: a NaN lies beyond every number on its sign's side,
 *     and between two NaNs the larger payload lies further out. */
static int f64_before(double x, double y, uint64_t bx, uint64_t by, uint64_t sign)
{
    int sx = (bx & sign) != 0, sy = (by & sign) != 0;
    if (sx != sy) {
#if ORACLE_MUTANT == 7
        if (x == y) return 0;                /* planted: -0 and +0 tie */
#endif
        return sx;
    }
    int nx = x != x, ny = y != y;
    if (!nx && !ny) return x < y;
    uint64_t mx = bx & ~sign, my = by & ~sign;
    if (nx && ny) return sx ? mx > my : mx < my;
    /* exactly one NaN: it lies outward on its side */
    return sx ? nx : ny;
}

static int typed_before(const void *x, const void *y, int type)
{
    switch (type) {
    case ORACLE_KEY_I32: return *(const int32_t *)x < *(const int32_t *)y;
    case ORACLE_KEY_U64: return *(const uint64_t *)x < *(const uint64_t *)y;
    case ORACLE_KEY_I64: return *(const int64_t *)x < *(const int64_t *)y;
    case ORACLE_KEY_F32: {
        float fx, fy;
        uint32_t bx, by;
        memcpy(&fx, x, 4); memcpy(&fy, y, 4); memcpy(&bx, x, 4); memcpy(&by, y, 4);
        /* the numbers compare exactly as doubles; the sign and the NaN
           payloads come from the float's own bits (placed in the top half),
           which the conversion cannot disturb */
        return f64_before(fx, fy, (uint64_t)bx << 32, (uint64_t)by << 32, 1ull << 63);
    }
    case ORACLE_KEY_F64: {
        double dx, dy;
        uint64_t bx, by;
        memcpy(&dx, x, 8); memcpy(&dy, y, 8); memcpy(&bx, x, 8); memcpy(&by, y, 8);
        return f64_before(dx, dy, bx, by, 1ull << 63);
    }
    }
    return 0;
}

static size_t typed_size(int type)
{
    return (type == ORACLE_KEY_I32 || type == ORACLE_KEY_F32) ? 4 : 8;
}

/* The last key of the type's order (pad value): the largest integer, or the
 * positive NaN with the largest payload. */
static void typed_max(unsigned char *out, int type)
{
    switch (type) {
    case ORACLE_KEY_I32: { int32_t v = INT32_MAX; memcpy(out, &v, 4); break; }
    case ORACLE_KEY_F32: { uint32_t v = 0x7FFFFFFFu; memcpy(out, &v, 4); break; }
    case ORACLE_KEY_U64: { uint64_t v = UINT64_MAX; memcpy(out, &v, 8); break; }
    case ORACLE_KEY_I64: { int64_t v = INT64_MAX; memcpy(out, &v, 8); break; }
    default:             { uint64_t v = 0x7FFFFFFFFFFFFFFFull; memcpy(out, &v, 8); break; }
    }
}

/* Section 3.1 network on keys of another type; same block directions, same
 * padding and descending reading as oracle_bitonic_sort_u32. */
int oracle_bitonic_sort_typed(void *keys, uint64_t n, int type, int ascending, oracle_counts *counts)
{
    oracle_counts local = {0, 0, 0};
    if (!counts) counts = &local;
    memset(counts, 0, sizeof(*counts));
    if (type < ORACLE_KEY_I32 || type > ORACLE_KEY_F64) return ORACLE_ERR_INVALID;
    if (n == 0) return ORACLE_OK;
    if (!keys) return ORACLE_ERR_INVALID;
    const size_t es = typed_size(type);
    uint64_t N = next_pow2_u64(n);
    unsigned char *a = (unsigned char *)malloc(N * es), tmp[8];
    if (!a) return ORACLE_ERR_NOMEM;
    memcpy(a, keys, n * es);
    for (uint64_t i = n; i < N; ++i) typed_max(a + i * es, type);
    int k = log2_u64(N);
    for (int p = 1; p <= k; ++p) {
        counts->phases += 1;
        for (int j = p - 1; j >= 0; --j) {
            uint64_t d = (uint64_t)1 << j;
            counts->steps += 1;
            for (uint64_t i = 0; i < N; ++i) {
                if (i & d) continue;
                unsigned char *x = a + i * es, *y = a + (i | d) * es;
                int up = block_ascending(i, p, k, ascending, 0);
                int out_of_order = up ? typed_before(y, x, type) : typed_before(x, y, type);
                if (out_of_order) {
                    memcpy(tmp, x, es);
                    memcpy(x, y, es);
                    memcpy(y, tmp, es);
                }
                counts->compare_exchanges += 1;
            }
        }
    }
    memcpy(keys, ascending ? a : a + (N - n) * es, n * es);
    free(a);
    return ORACLE_OK;
}

int oracle_mutant_id(void) { return ORACLE_MUTANT; }
