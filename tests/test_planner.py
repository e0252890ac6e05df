"""Host-side tests of the launch planner: every plan is executed by a numpy
emulation of the tile kernel (tests/plan_emulator.py) and compared with the
oracle.  No GPU: the library is only asked for descriptors.
"""
import numpy as np
import pytest

import oracle
import paper_1506_01446_gb300 as bt
import workloads
from plan_emulator import Stats, debug_plan, emulate

pytestmark = pytest.mark.skipif(not __import__("os").path.exists(bt.LIB_PATH),
                                reason="CUDA library not built")


@pytest.fixture(autouse=True)
def default_options():
    bt.set_options(variant=0, tile_log2=0, global_bits=0, use_graph=1, keys_per_thread_log2=0, min_row_log2=0,
                   ctas_per_sm=0)
    yield
    bt.set_options(variant=0, tile_log2=0, global_bits=0, use_graph=1, keys_per_thread_log2=0, min_row_log2=0,
                   ctas_per_sm=0)


SIZES = [2, 3, 17, 4095, 4096, 8193, 16384, 16385, 70001, 1 << 17]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("ascending", [True, False])
def test_keys_plan_sorts(n, ascending):
    keys = workloads.uniform_u32(n, seed=n)
    for front in (0, 1, 3):
        st = Stats()
        got, plan, st = emulate(keys, ascending, front, st)
        want, _ = oracle.bitonic_sort(keys, ascending)
        assert np.array_equal(got, want), (n, front)
        assert st.conflicted_quarter_warps == 0
        assert st.uncoalesced_rounds == 0


@pytest.mark.parametrize("variant,tile", [(0, 13), (2, 0), (1, 0), (0, 14)])
def test_other_variants_and_tiles(variant, tile):
    bt.set_options(variant=variant, tile_log2=tile)
    for n in (1000, 40000, 1 << 16):
        for dist in ("uniform", "distinct16", "reverse"):
            keys = workloads.keys_u32(dist, n, seed=3)
            got, _, _ = emulate(keys, True, 0)
            assert np.array_equal(got, oracle.merge_sort(keys)), (variant, tile, n, dist)


@pytest.mark.parametrize("tile,kpt,cap", [(14, 6, 0), (14, 6, 3), (14, 5, 0), (13, 5, 0)])
def test_tile_configurations(tile, kpt, cap):
    bt.set_options(tile_log2=tile, keys_per_thread_log2=kpt, ctas_per_sm=cap)
    # configuration ids: 0 = 256 x 64 bounded for two CTAs (the default), 7 =
    # capped for three, 2 = 512 x 32, 1 = 8K keys as 256 x 32
    expect_cfg = {(14, 6, 0): 0, (14, 6, 3): 7, (14, 5, 0): 2, (13, 5, 0): 1}[(tile, kpt, cap)]
    for n in (3000, 1 << 17):
        keys = workloads.uniform_u32(n, seed=kpt)
        assert debug_plan(n, 4)["cfg"] == expect_cfg
        got, _, st = emulate(keys, True, 1)
        assert np.array_equal(got, oracle.merge_sort(keys)), (tile, kpt, n)
        assert st.conflicted_quarter_warps == 0
    comp = np.arange(70001, dtype=np.uint64)[::-1].copy()
    bt.set_options(tile_log2=0, keys_per_thread_log2=0)
    got, _, _ = emulate(comp, True, 0)
    assert np.array_equal(got, np.sort(comp))


@pytest.mark.parametrize("io_direct", [1, 2, 3])
def test_direct_io_layouts(io_direct):
    bt.set_options(io_direct=io_direct)
    for n in (5000, (1 << 18) + 1):
        keys = workloads.uniform_u32(n, seed=io_direct)
        got, _, st = emulate(keys, False, 2)
        assert np.array_equal(got, oracle.merge_sort(keys, False))
    bt.set_options(io_direct=0)


@pytest.mark.parametrize("row", [3, 4, 6])
def test_min_row_lengths(row):
    bt.set_options(min_row_log2=row)
    for n in (70001, (1 << 19) + 3):
        keys = workloads.uniform_u32(n, seed=row)
        got, plan, st = emulate(keys, True, 1)
        assert np.array_equal(got, oracle.merge_sort(keys))
        assert st.conflicted_quarter_warps == 0
    comp = np.arange(100003, dtype=np.uint64)[::-1].copy()
    got, _, _ = emulate(comp, True, 0)
    assert np.array_equal(got, np.sort(comp))
    bt.set_options(min_row_log2=0)


@pytest.mark.parametrize("gb", [1, 2, 3, 5, 9])
def test_global_bits_choices(gb):
    bt.set_options(global_bits=gb)
    keys = workloads.uniform_u32((1 << 18) + 5, seed=gb)
    got, plan, _ = emulate(keys, False, 2)
    assert np.array_equal(got, oracle.merge_sort(keys, False))


@pytest.mark.parametrize("n", [3, 1000, 8192, 8193, 50000])
def test_composite_plan_sorts(n):
    # 64-bit composites (key << 32 | index), the pair sort's working array
    keys = (workloads.uniform_u32(n, seed=n) >> np.uint32(24)).astype(np.uint64)
    comp = (keys << np.uint64(32)) | np.arange(n, dtype=np.uint64)
    # (tile, keys per thread): 8K composites as 256 x 32 (default), 4K as 256 x 16
    for tile, kpt in ((0, 0), (12, 0)):
        bt.set_options(tile_log2=tile, keys_per_thread_log2=kpt)
        got, _, st = emulate(comp, True, 0)
        assert np.array_equal(got, np.sort(comp))
        assert st.conflicted_quarter_warps == 0


def test_plan_counts_match_section_3_2():
    # Every plan runs exactly the k(k+1)/2 steps of the network (Section 3.2).
    for k in (10, 14, 16, 20, 24, 28, 31):
        for variant in (0, 1, 2):
            bt.set_options(variant=variant)
            info = bt.plan_info(1 << k)
            assert info["fused_steps"] + info["global_steps"] == k * (k + 1) // 2, (k, variant)
    bt.set_options(variant=1)
    assert bt.plan_info(1 << 20)["launches"] == 20 * 21 // 2   # Section 3.3: one kernel per step


def test_plan_info_headline_size():
    info = bt.plan_info(1 << 28)
    assert info["hbm_passes"] == info["launches"]
    assert info["hbm_passes"] <= 40


def test_split_weighs_transposes():
    # The optimized plan splits the steps into passes by cost (one pass = a
    # read and a write of every key; one transpose = a shared-memory round
    # trip inside a pass).  At 2^28 4-byte keys the greedy longest-pass split
    # needs 27 passes and 82 transposes; the weighted split trades one pass
    # for twelve transposes.
    bt.set_options(variant=0, global_bits=8)
    P = debug_plan(1 << 28, 4)
    transposes = sum(int(P["descs"][L[5]]["nrounds"]) - 1 for L in P["launches"])
    assert len(P["launches"]) <= 28
    assert 4 * len(P["launches"]) + transposes <= 4 * 27 + 82 - 8
    assert transposes <= 70


def test_debug_plan_follows_class_options():
    # bitonic_debug_plan reports the plan the sort itself would run: a size
    # class's tuned options (here 8K-key tiles for 2^20 keys) apply to that
    # class only
    bt.set_options(tile_log2=0, keys_per_thread_log2=0, ctas_per_sm=0)
    try:
        bt.set_class_options(4, 20, dict(tile_log2=13, keys_per_thread_log2=5, l2_prefetch=1))
        assert debug_plan(1 << 20, 4)["cfg"] == 1
        assert debug_plan((1 << 19) + 1, 4)["cfg"] == 1
        assert debug_plan(1 << 21, 4)["cfg"] == 0
        assert debug_plan(1 << 20, 8)["cfg"] == 4
    finally:
        bt.set_class_options(4, 20, None)
    assert debug_plan(1 << 20, 4)["cfg"] == 0


def test_round_shapes_cover_every_step():
    # The descriptors' register rounds hold every step of the network once:
    # k(k+1)/2 steps for 2^k keys (Section 3.2), 105 of them (phases 1..14)
    # in the tile sort, and every launch of the optimized plan at 2^28 is a
    # tile pass of at most 14 steps after it.
    bt.set_options(variant=0, tile_log2=0, keys_per_thread_log2=0, ctas_per_sm=0, global_bits=0)
    for k, kb in ((16, 4), (20, 4), (28, 4), (20, 8), (26, 8)):
        shapes = bt.round_shapes(bt.debug_plan(1 << k, kb))
        assert sum(sum(s) for s in shapes) == k * (k + 1) // 2, (k, kb)
    shapes = bt.round_shapes(bt.debug_plan(1 << 28, 4))
    assert sum(shapes[0]) == 14 * 15 // 2
    assert all(sum(s) <= 14 for s in shapes[1:])
    assert len(shapes) == bt.plan_info(1 << 28)["launches"]


def test_graph_kernels_count_the_split_ranges():
    # A graph-captured sort splits every run of at least two launches whose
    # strides stay below bit k - split_log2 into 2^split_log2 tile ranges,
    # one kernel each; the plan itself is unchanged.
    saved = bt.get_options()
    try:
        for split in (0, 1, 2):
            bt.set_options(split_log2=split)
            for k in (16, 20, 24, 28):
                plan = bt.debug_plan(1 << k)
                his = [la[2] for la in plan["launches"]]
                his_ok = [h < k - split and (1 << (k - 14)) % (1 << split) == 0 and (1 << (k - 14)) >= 256
                          for h in his]
                want, i = 0, 0
                while i < len(his):
                    j = i
                    while split and j < len(his) and his_ok[j]:
                        j += 1
                    if j - i >= 2:
                        want += (j - i) << split
                        i = j
                    else:
                        want += 1
                        i += 1
                assert bt.graph_kernels(1 << k) == want, (split, k)
                assert bt.plan_info(1 << k)["launches"] == len(his)
        bt.set_options(split_log2=1)
        assert bt.graph_kernels(1 << 28) == 55 and bt.plan_info(1 << 28)["launches"] == 28
    finally:
        bt.set_options(**saved)
