"""Seeded synthetic inputs shared by the oracle tests, the GPU parity tests and
the benchmark.

This module only draws numbers: it holds none of the sorting network's
arithmetic and never orders anything (the "already sorted" distribution is
built as a running sum of non-negative increments, not by sorting).

Every generator is a pure function of its arguments.  Randomness comes from
splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output i of stream ``seed`` is
``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``; a 32-bit key is the high half of
a 64-bit output, a float in [0, 1) is its top 53 bits.

The workload shapes follow the paper's experiments (Section 5: random 32-bit
integers, 128K to 256M keys) widened to the distributions, key/value pairs,
segment mixes and request streams the library supports.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

ALL_EQUAL_VALUE = 0x9E3779B9

# Default seeds of the named workloads (any seed may be passed explicitly).
SEEDS = {
    "key_types": 1506_01446_6,
    "n16_uniform": 1506_01446,
    "n24": 2024,
    "n24_npow2": 10_000_019,
    "n28_uniform": 28,
    "pairs_n26": 26,
    "segmented": 65536,
    "serving": 20000,
}

DISTRIBUTIONS = ("uniform", "sorted", "reverse", "all_equal", "distinct16")


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of splitmix64 stream ``seed`` (uint64)."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + i * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _chunked_u32(seed: int, n: int, chunk: int = 1 << 24) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    for s in range(0, n, chunk):
        c = min(chunk, n - s)
        out[s:s + c] = (splitmix64(seed, c, start=s) >> np.uint64(32)).astype(np.uint32)
    return out


def uniform_u32(n: int, seed: int) -> np.ndarray:
    """n keys uniform over [0, 2^32)."""
    return _chunked_u32(seed, n)


def uniform01(n: int, seed: int) -> np.ndarray:
    """n doubles uniform over [0, 1)."""
    z = splitmix64(seed, n)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def keys_u32(dist: str, n: int, seed: int) -> np.ndarray:
    """One of the five key distributions of the 2^24-key workload."""
    if dist == "uniform":
        return uniform_u32(n, seed)
    if dist in ("sorted", "reverse"):
        # Non-decreasing by construction: a running sum of increments drawn in
        # [0, 2 * 2^32 / n), clipped to the 32-bit range.
        if n == 0:
            return np.empty(0, dtype=np.uint32)
        step = max(1, (2 << 32) // max(n, 1))
        inc = (splitmix64(seed, n) % np.uint64(step)).astype(np.uint64)
        run = np.minimum(np.cumsum(inc, dtype=np.uint64), np.uint64(0xFFFFFFFF))
        out = run.astype(np.uint32)
        return out if dist == "sorted" else out[::-1].copy()
    if dist == "all_equal":
        return np.full(n, ALL_EQUAL_VALUE, dtype=np.uint32)
    if dist == "distinct16":
        vals = (splitmix64(seed ^ 0x5EED, 64) >> np.uint64(32)).astype(np.uint32)
        vals = np.array(list(dict.fromkeys(vals.tolist()))[:16], dtype=np.uint32)
        pick = (splitmix64(seed, n) >> np.uint64(60)).astype(np.int64)  # 0..15
        return vals[pick]
    raise ValueError(f"unknown distribution {dist!r}")


def pair_keys_u32(n: int, seed: int, key_bits: int = 20) -> tuple[np.ndarray, np.ndarray]:
    """Key/value workload: keys uniform over [0, 2^key_bits) (many ties),
    values = original index."""
    k = (uniform_u32(n, seed) >> np.uint32(32 - key_bits)).astype(np.uint32) if key_bits < 32 \
        else uniform_u32(n, seed)
    v = np.arange(n, dtype=np.uint32)
    return k, v


def segment_lengths(nseg: int, seed: int, max_len: int = 8192, min_len: int = 1) -> np.ndarray:
    """Lengths log-uniform in [min_len, max_len]:
    clamp(floor(min_len * exp(U * ln((max_len + 1) / min_len))), min_len, max_len)."""
    u = uniform01(nseg, seed)
    lens = np.floor(min_len * np.exp(u * np.log((max_len + 1) / min_len))).astype(np.int64)
    return np.clip(lens, min_len, max_len)


def segmented_u32(nseg: int, seed: int, max_len: int = 8192) -> tuple[np.ndarray, np.ndarray]:
    """Contiguous keys of ``nseg`` segments plus int32 CSR offsets (nseg + 1)."""
    lens = segment_lengths(nseg, seed, max_len)
    offs = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    keys = uniform_u32(int(offs[-1]), seed ^ 0xC0FFEE)
    return keys, offs.astype(np.int32)


def serving_requests(count: int, seed: int, rate: float = 2000.0, lo_log2: int = 10,
                     hi_log2: int = 22, pair_frac: float = 0.3):
    """Request stream: Poisson arrivals at ``rate``/s, sizes log-uniform in
    [2^lo_log2, 2^hi_log2], a ``pair_frac`` share carrying values.

    Returns (arrival_s float64[count], sizes int64[count], has_vals bool[count]).
    """
    u_gap = uniform01(count, seed)
    gaps = -np.log1p(-u_gap) / rate
    arrival = np.cumsum(gaps)
    u_sz = uniform01(count, seed ^ 0xABCDEF)
    lo, hi = 2.0 ** lo_log2, 2.0 ** hi_log2
    sizes = np.floor(lo * np.exp(u_sz * np.log((hi + 1) / lo))).astype(np.int64)
    sizes = np.clip(sizes, int(lo), int(hi))
    has_vals = uniform01(count, seed ^ 0x123457) < pair_frac
    return arrival, sizes, has_vals


TYPED_KEY_KINDS = ("int32", "float32", "uint64", "int64", "float64")

# Bit patterns every typed test mixes in: integer extremes; for floats the
# signed zeros, infinities, subnormals and NaNs of both signs and kinds with
# several payloads.
_SPECIAL_BITS = {
    "int32": [0x80000000, 0x80000001, 0xFFFFFFFF, 0, 1, 0x7FFFFFFE, 0x7FFFFFFF],
    "float32": [0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x00000001, 0x80000001, 0x007FFFFF,
                0x7FC00000, 0xFFC00000, 0x7F800001, 0xFF800001, 0x7FFFFFFF, 0xFFFFFFFF, 0x7FC00123],
    "uint64": [0, 1, 0x7FFFFFFFFFFFFFFF, 0x8000000000000000, 0xFFFFFFFFFFFFFFFF, 0xFFFFFFFF, 0x100000000],
    "int64": [0x8000000000000000, 0xFFFFFFFFFFFFFFFF, 0, 1, 0x7FFFFFFFFFFFFFFF],
    "float64": [0, 0x8000000000000000, 0x7FF0000000000000, 0xFFF0000000000000, 1, 0x8000000000000001,
                0x7FF8000000000000, 0xFFF8000000000000, 0x7FF0000000000001, 0xFFF0000000000001,
                0x7FFFFFFFFFFFFFFF, 0xFFFFFFFFFFFFFFFF],
}
_TYPED_DTYPES = {"int32": (np.int32, np.uint32), "float32": (np.float32, np.uint32),
                 "uint64": (np.uint64, np.uint64), "int64": (np.int64, np.uint64),
                 "float64": (np.float64, np.uint64)}


def typed_keys(kind: str, n: int, seed: int, specials: bool = True) -> np.ndarray:
    """n keys of a numpy dtype from uniform random bit patterns (for floats
    that spans every binade, with a few NaNs and infinities).  specials:
    scatter the kind's special bit patterns through the array (about 1 in 16
    keys).  specials=False gives keys on which numpy's order is the type's
    total order: no NaNs and no negative zeros (replaced by 1.0 and +0)."""
    dt, bits = _TYPED_DTYPES[kind]
    z = splitmix64(seed, n)
    raw = (z >> np.uint64(32)).astype(np.uint32) if np.dtype(bits).itemsize == 4 else z
    raw = raw.astype(bits)
    if specials:
        sp = np.array(_SPECIAL_BITS[kind], dtype=np.uint64).astype(bits)
        pick = splitmix64(seed + 1, n)
        where = (pick & np.uint64(15)) == 0
        raw[where] = sp[(pick[where] >> np.uint64(8)) % np.uint64(sp.size)]
    keys = raw.view(dt).copy()
    if not specials and np.dtype(dt).kind == "f":
        keys[np.isnan(keys)] = dt(1.0)
        keys[(keys == 0) & np.signbit(keys)] = dt(0.0)
    return keys
