// Catalog of round patterns compiled as straight-line code (host + device).
//
// A round's steps, in register-index bits, always have the shape
//   [full sort of register bits 0..s-1]            (phases 1..s, Section 3.1)
//   [half-cleaners at bits a, a-1, ..., b]
//   [mirror step at bit f, half-cleaners f-1, ..., c]
// Rounds whose steps match a catalog entry run that entry's unrolled code;
// any other round falls back to the per-step dispatcher.
#pragma once

#include <stdint.h>

#include "desc.h"

namespace bitonic {

constexpr int kMaxPatternSteps = 28;
constexpr uint8_t kGenericPattern = 0xFF;

struct RoundPattern {
    int n;
    uint8_t steps[kMaxPatternSteps];
};

// Structural description: s = full-sort phases (0 = none); halves a..b
// (a < 0 = none); mirror step at f then halves f-1..c (f < 0 = none).
struct PatternSpec {
    int s, a, b, f, c;
};

constexpr RoundPattern build_pattern(PatternSpec p)
{
    RoundPattern r{0, {}};
    for (int q = 1; q <= p.s; ++q) {
        r.steps[r.n++] = (uint8_t)((q - 1) | kStepFlip);
        for (int h = q - 2; h >= 0; --h) r.steps[r.n++] = (uint8_t)h;
    }
    if (p.a >= 0)
        for (int h = p.a; h >= p.b; --h) r.steps[r.n++] = (uint8_t)h;
    if (p.f >= 0) {
        r.steps[r.n++] = (uint8_t)(p.f | kStepFlip);
        for (int h = p.f - 1; h >= p.c; --h) r.steps[r.n++] = (uint8_t)h;
    }
    return r;
}

// Catalog for 64 keys per thread (4-byte keys: vector bits 0..1) and for 32
// composites per thread (8-byte keys: vector bit 0): the shapes the planner
// produces for the default tile configurations.
constexpr PatternSpec kCatalogR6[] = {
    {0, -1, 0, -1, 0},                                    // no steps (coalescing round)
    {0, 5, 2, -1, 0}, {0, 5, 0, -1, 0}, {0, 4, 2, -1, 0}, {0, 4, 0, -1, 0}, {0, 3, 2, -1, 0},
    {0, 3, 0, -1, 0}, {0, 2, 2, -1, 0}, {0, 2, 0, -1, 0},
    {0, -1, 0, 5, 2}, {0, -1, 0, 5, 3}, {0, -1, 0, 5, 4}, {0, -1, 0, 5, 5},
    {0, 2, 0, 5, 3}, {0, 3, 0, 5, 4}, {0, 4, 0, 5, 5}, {0, 2, 0, 5, 2},
    {6, -1, 0, -1, 0}, {5, -1, 0, -1, 0},
};
constexpr PatternSpec kCatalogR5[] = {
    {0, -1, 0, -1, 0},
    {0, 4, 1, -1, 0}, {0, 4, 0, -1, 0}, {0, 4, 2, -1, 0}, {0, 3, 2, -1, 0}, {0, 3, 0, -1, 0},
    {0, 3, 3, -1, 0}, {0, 2, 1, -1, 0}, {0, 2, 0, -1, 0}, {0, 1, 1, -1, 0}, {0, 1, 0, -1, 0},
    {0, -1, 0, 4, 1}, {0, -1, 0, 4, 2}, {0, -1, 0, 4, 3}, {0, -1, 0, 4, 4},
    {0, 1, 0, 4, 2}, {0, 2, 0, 4, 3}, {0, 3, 0, 4, 4}, {0, 2, 0, 4, 4}, {0, 1, 0, 4, 1},
    {5, -1, 0, -1, 0}, {4, -1, 0, -1, 0},
};
constexpr int kCatalogR6Size = sizeof(kCatalogR6) / sizeof(kCatalogR6[0]);
constexpr int kCatalogR5Size = sizeof(kCatalogR5) / sizeof(kCatalogR5[0]);

// Catalog used by a kernel with 2^LOG_R keys per thread (empty for others).
constexpr int catalog_size(int log_r) { return log_r == 6 ? kCatalogR6Size : (log_r == 5 ? kCatalogR5Size : 0); }

constexpr PatternSpec catalog_spec(int log_r, int i)
{
    return log_r == 6 ? kCatalogR6[i] : kCatalogR5[i];
}

constexpr RoundPattern catalog_pattern(int log_r, int i) { return build_pattern(catalog_spec(log_r, i)); }

}  // namespace bitonic
