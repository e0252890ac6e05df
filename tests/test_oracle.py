"""Pins for the CPU oracle: checks it against what the paper and mathematics
fix, not against itself.

  - the worked bitonic sequences of Section 3.1 (tests/golden/paper_section3.txt)
  - the step / compare-exchange closed forms of Sections 3.1-3.3
  - the 0-1 principle (Knuth TAOCP vol. 3, 5.3.4), exhaustive for m <= 16
  - agreement with numpy's sort / stable argsort (library special case)
  - multiset and sortedness invariants
  - each planted mistake in the oracle (ORACLE_MUTANT builds) fails a pin
"""
import numpy as np
import pytest

import oracle
import workloads
from conftest import read_golden


def is_bitonic(seq):
    """Definition of Section 3.1: some cyclic rotation rises then falls."""
    n = len(seq)
    for r in range(max(n, 1)):
        s = list(seq[r:]) + list(seq[:r])
        i = 0
        while i + 1 < n and s[i] <= s[i + 1]:
            i += 1
        while i + 1 < n and s[i] >= s[i + 1]:
            i += 1
        if i >= n - 1:
            return True
    return False


def golden():
    return read_golden("paper_section3.txt")


def test_worked_sequences_are_bitonic():
    seqs = [list(map(int, s)) for s in golden()["bitonic_sequence"]]
    assert len(seqs) == 2
    for s in seqs:
        assert is_bitonic(s)
    # the second is a rotation of the first (Section 3.1)
    a, b = seqs
    assert any(a[r:] + a[:r] == b for r in range(len(a)))


@pytest.mark.parametrize("which", [0, 1])
def test_half_cleaner_on_worked_sequences(which):
    seq = np.array(list(map(int, golden()["bitonic_sequence"][which])), dtype=np.uint32)
    n = seq.size
    one = oracle.bitonic_merge(seq, ascending=True, max_steps=1)
    lo, hi = one[: n // 2], one[n // 2:]
    # Batcher's half-cleaner lemma: both halves bitonic, every low <= every high
    assert is_bitonic(lo.tolist()) and is_bitonic(hi.tolist())
    assert lo.max() <= hi.min()
    assert sorted(one.tolist()) == sorted(seq.tolist())
    full = oracle.bitonic_merge(seq, ascending=True)
    assert full.tolist() == sorted(seq.tolist())
    full_desc = oracle.bitonic_merge(seq, ascending=False)
    assert full_desc.tolist() == sorted(seq.tolist(), reverse=True)


def test_network_n8_counts_from_section_3_1():
    g = dict(kv.split("=") for kv in golden()["network_n8"][0])
    _, c = oracle.bitonic_sort(np.arange(8, dtype=np.uint32)[::-1])
    assert c.phases == int(g["phases"])
    assert c.steps == int(g["steps"])
    assert c.compare_exchanges == int(g["compare_exchanges"])
    assert c.compare_exchanges // c.steps == int(g["per_step"])


@pytest.mark.parametrize("k", list(range(0, 21)))
def test_counts_match_section_3_2_closed_forms(k):
    n = 1 << k
    keys = workloads.uniform_u32(n, seed=k)
    out, c = oracle.bitonic_sort(keys)
    # Section 3.2: log n (log n + 1) / 2 rounds and n log n (log n + 1) / 4
    # compare-exchanges; Section 3.3: N/2 compare-exchanges per round.
    assert c.phases == k
    assert c.steps == k * (k + 1) // 2
    assert c.compare_exchanges == n * k * (k + 1) // 4
    if k:
        assert c.compare_exchanges == c.steps * (n // 2)
    assert np.array_equal(out, np.sort(keys))


@pytest.mark.parametrize("n", [3, 5, 6, 7, 9, 1000, 4097])
def test_counts_for_padded_sizes(n):
    N = 1 << (n - 1).bit_length()
    k = N.bit_length() - 1
    _, c = oracle.bitonic_sort(workloads.uniform_u32(n, seed=n))
    assert c.steps == k * (k + 1) // 2
    assert c.compare_exchanges == N * k * (k + 1) // 4


@pytest.mark.parametrize("ascending", [True, False])
@pytest.mark.parametrize("first_descending", [False, True])
def test_zero_one_principle_exhaustive(ascending, first_descending):
    for m in range(0, 17):
        assert oracle.zero_one_failures(m, ascending, first_descending) == 0, m


SIZES = [0, 1, 2, 3, 4, 7, 8, 9, 31, 32, 33, 255, 1000, 4096, 4097, 65539]


@pytest.mark.parametrize("dist", workloads.DISTRIBUTIONS)
@pytest.mark.parametrize("ascending", [True, False])
def test_network_equals_library_sort(dist, ascending):
    for n in SIZES:
        keys = workloads.keys_u32(dist, n, seed=7 + n)
        want = np.sort(keys) if ascending else np.sort(keys)[::-1]
        got, _ = oracle.bitonic_sort(keys, ascending)
        assert np.array_equal(got, want), (dist, n)
        got2, _ = oracle.bitonic_sort(keys, ascending, first_descending=True)
        assert np.array_equal(got2, want), (dist, n)
        assert np.array_equal(oracle.merge_sort(keys, ascending), want), (dist, n)
        if ascending:
            assert np.array_equal(oracle.quicksort(keys), want), (dist, n)


def test_sentinel_valued_keys_with_padding():
    # real 0xFFFFFFFF keys mixed with the pad value at a non-power-of-two size
    for n in [3, 5, 13, 1023, 1025]:
        keys = workloads.uniform_u32(n, seed=n)
        keys[::3] = 0xFFFFFFFF
        keys[1::7] = 0
        for asc in (True, False):
            want = np.sort(keys) if asc else np.sort(keys)[::-1]
            got, _ = oracle.bitonic_sort(keys, asc)
            assert np.array_equal(got, want)


def stable_order(keys, ascending):
    idx = np.arange(keys.size)
    k = keys.astype(np.int64)
    return np.lexsort((idx, k if ascending else -k))


@pytest.mark.parametrize("ascending", [True, False])
def test_pairs_tie_order_by_index(ascending):
    for n in [0, 1, 2, 5, 64, 1000, 4099]:
        keys = (workloads.uniform_u32(n, seed=n) >> np.uint32(28)).astype(np.uint32)  # 16 values
        vals = workloads.uniform_u32(n, seed=n + 1)
        order = stable_order(keys, ascending)
        k1, v1, c = oracle.bitonic_sort_pairs(keys, vals, ascending)
        assert np.array_equal(k1, keys[order]) and np.array_equal(v1, vals[order]), n
        k2, v2 = oracle.merge_sort_pairs(keys, vals, ascending)
        assert np.array_equal(k2, keys[order]) and np.array_equal(v2, vals[order]), n
        if n:
            N = 1 << (n - 1).bit_length()
            kk = N.bit_length() - 1
            assert c.compare_exchanges == N * kk * (kk + 1) // 4


def test_pairs_with_index_values_satisfy_identity():
    keys, vals = workloads.pair_keys_u32(5000, seed=3, key_bits=8)
    k, v, _ = oracle.bitonic_sort_pairs(keys, vals)
    assert np.array_equal(k, keys[v])                 # out_key[i] == in_key[out_val[i]]
    same = k[1:] == k[:-1]
    assert np.all(v[1:][same] > v[:-1][same])          # ties by increasing index


def test_segmented_equals_per_segment_sort():
    keys, offs = workloads.segmented_u32(200, seed=5, max_len=300)
    got = oracle.segmented_sort(keys, offs)
    want = keys.copy()
    for s in range(offs.size - 1):
        want[offs[s]:offs[s + 1]] = np.sort(keys[offs[s]:offs[s + 1]])
    assert np.array_equal(got, want)
    vals = np.arange(keys.size, dtype=np.uint32)
    gk, gv = oracle.segmented_sort_pairs(keys, vals, offs)
    for s in range(offs.size - 1):
        a, b = offs[s], offs[s + 1]
        o = stable_order(keys[a:b], True)
        assert np.array_equal(gk[a:b], keys[a:b][o]) and np.array_equal(gv[a:b], vals[a:b][o])


def test_checkers():
    a = workloads.uniform_u32(1000, seed=1)
    s = np.sort(a)
    assert oracle.is_sorted(s) and not oracle.is_sorted(a)
    assert oracle.is_sorted(s[::-1], ascending=False)
    assert oracle.same_multiset(a, s)
    b = s.copy()
    b[10] ^= 1
    assert not oracle.same_multiset(a, b)


def test_input_generators_shapes():
    keys, offs = workloads.segmented_u32(65536, seed=workloads.SEEDS["segmented"])
    lens = np.diff(offs)
    assert lens.min() >= 1 and lens.max() <= 8192
    assert 55e6 < keys.size < 65e6                      # ~59.6M keys in all
    for d in workloads.DISTRIBUTIONS:
        k = workloads.keys_u32(d, 1 << 12, seed=1)
        assert k.dtype == np.uint32 and k.size == 1 << 12
    assert np.all(np.diff(workloads.keys_u32("sorted", 4096, 3).astype(np.int64)) >= 0)
    assert len(np.unique(workloads.keys_u32("distinct16", 4096, 3))) == 16
    arr, sizes, hv = workloads.serving_requests(20000, seed=1)
    assert np.all(np.diff(arr) > 0) and sizes.min() >= 1024 and sizes.max() <= 1 << 22
    assert 0.25 < hv.mean() < 0.35


TYPED = {"f32": (np.float32, np.uint32), "f64": (np.float64, np.uint64), "i32": (np.int32, np.uint32),
         "i64": (np.int64, np.uint64), "u64": (np.uint64, np.uint64)}


def golden_order(name):
    """Ascending keys of one golden line, as an array of the key type."""
    dt, bits = TYPED[name]
    (vals,) = read_golden("ieee754_total_order.txt")["order_" + name]
    return np.array([int(v, 16) for v in vals], dtype=bits).view(dt)


def check_golden_order(name, lib=None):
    a = golden_order(name)
    _, bits = TYPED[name]
    for seed in range(3):
        rng = np.random.default_rng(seed)
        counts = rng.integers(1, 4, size=a.size)
        want = np.repeat(a, counts)
        x = want[rng.permutation(want.size)]
        up = oracle.bitonic_sort_typed(x, True, lib=lib)[0]
        down = oracle.bitonic_sort_typed(x, False, lib=lib)[0]
        if not (np.array_equal(up.view(bits), want.view(bits)) and
                np.array_equal(down.view(bits), want[::-1].view(bits))):
            return False
    return True


def pin_battery(lib):
    """Returns the names of pins that fail for the oracle library ``lib``."""
    failed = []
    if not check_golden_order("f32", lib) or not check_golden_order("f64", lib):
        failed.append("ieee_total_order")
    for m in (4, 5, 8):
        if oracle.zero_one_failures(m, True, lib=lib) or oracle.zero_one_failures(m, False, lib=lib):
            failed.append(f"zero_one_{m}")
    _, c = oracle.bitonic_sort(np.arange(16, dtype=np.uint32), lib=lib)
    if c.steps != 10 or c.compare_exchanges != 16 * 4 * 5 // 4:
        failed.append("counts")
    keys = workloads.uniform_u32(777, seed=9)
    if not np.array_equal(oracle.bitonic_sort(keys, lib=lib)[0], np.sort(keys)):
        failed.append("library")
    tk = (keys >> np.uint32(29)).astype(np.uint32)
    tv = np.arange(tk.size, dtype=np.uint32)
    o = stable_order(tk, True)
    if not np.array_equal(oracle.bitonic_sort_pairs(tk, tv, lib=lib)[1], tv[o]):
        failed.append("pairs_network")
    if not np.array_equal(oracle.merge_sort_pairs(tk, tv, lib=lib)[1], tv[o]):
        failed.append("pairs_merge")
    return failed


def test_pin_battery_passes_on_the_oracle():
    assert pin_battery(oracle.load()) == []


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6, 7])
def test_planted_mistakes_are_caught(mutant, tmp_path):
    lib = oracle.load(mutant=mutant, out_dir=str(tmp_path))
    assert lib.oracle_mutant_id() == mutant
    assert pin_battery(lib), f"mutant {mutant} passed every pin"


@pytest.mark.parametrize("name", sorted(TYPED))
def test_typed_orders_from_definitions(name):
    # IEEE 754-2008 clause 5.10 (floats) and two's-complement / unsigned
    # numeric order (integers), written out in tests/golden.
    assert check_golden_order(name)


@pytest.mark.parametrize("name", sorted(TYPED))
@pytest.mark.parametrize("n", [1, 2, 3, 100, 1000, 4097])
def test_typed_network_equals_library_sort(name, n):
    # Without NaNs and negative zeros, every type's order is numpy's.
    dt, bits = TYPED[name]
    rng = np.random.default_rng(n)
    raw = rng.integers(0, 2**63, size=n, dtype=np.uint64) * 2 + rng.integers(0, 2, size=n, dtype=np.uint64)
    x = raw.astype(bits).view(dt) if np.dtype(bits).itemsize == 8 else (raw >> np.uint64(32)).astype(bits).view(dt)
    if np.dtype(dt).kind == "f":
        x = np.where(np.isnan(x) | ((x == 0) & np.signbit(x)), dt(1.25), x).astype(dt)
        x[:: 7] = np.inf
        x[3:: 11] = -np.inf
    for asc in (True, False):
        got, c = oracle.bitonic_sort_typed(x, asc)
        want = np.sort(x) if asc else np.sort(x)[::-1]
        assert np.array_equal(got.view(bits), want.view(bits)), (name, n, asc)
        N = 1 << max(0, (n - 1).bit_length())
        k = N.bit_length() - 1
        assert c.compare_exchanges == N * k * (k + 1) // 4    # Section 3.2


def test_typed_rejects_other_types():
    with pytest.raises(TypeError):
        oracle.bitonic_sort_typed(np.arange(4, dtype=np.int16))


def test_cpu_comparison_sorts():
    # The benchmark's CPU references (std::sort on one core; one std::sort per
    # thread, then parallel merges) and the Section 5 quicksort agree with
    # numpy's sort on seeded inputs, ragged sizes and thread counts included.
    for n in (0, 1, 2, 3, 17, 1000, 65537, (1 << 20) + 3):
        keys = workloads.uniform_u32(n, seed=n + 21)
        keys[::5] = keys[0] if n else keys[::5]
        want = np.sort(keys)
        assert np.array_equal(oracle.std_sort(keys), want)
        assert np.array_equal(oracle.quicksort(keys), want)
        for threads in (1, 2, 3, 7, 16):
            assert np.array_equal(oracle.parallel_sort(keys, threads), want), (n, threads)
