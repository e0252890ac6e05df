"""GPU parity: the CUDA path through the C ABI, bit-exact against the CPU
oracle on seeded inputs (sorting has a unique result, so no tolerance)."""
import os

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1506_01446_gb300 as bt  # noqa: E402


def to_dev(a: np.ndarray, pad_front: int = 0):
    """uint32 numpy -> int32 CUDA tensor view (same bits); optional leading
    elements make the returned view start 4*pad_front bytes past a 16-byte
    boundary."""
    buf = np.zeros(a.size + pad_front, dtype=np.uint32)
    buf[pad_front:] = a
    t = torch.from_numpy(buf.view(np.int32)).cuda()
    return t[pad_front:]


def to_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


LIBRARY_DEFAULTS = bt.get_options() if os.path.exists(bt.LIB_PATH) else {}


@pytest.fixture(autouse=True)
def default_options():
    bt.set_options(**LIBRARY_DEFAULTS)
    yield
    bt.set_options(**LIBRARY_DEFAULTS)
    assert bt.last_device_error() == bt.OK


def check_keys(keys, ascending=True, pad_front=0):
    t = to_dev(keys, pad_front)
    bt.sort_(t, ascending)
    torch.cuda.synchronize()
    got = to_host(t)
    want = oracle.merge_sort(keys, ascending)
    assert np.array_equal(got, want), f"n={keys.size} asc={ascending} front={pad_front}"


EDGE_SIZES = [0, 1, 2, 3, 4, 5, 7, 8, 31, 33, 1000, 4095, 4096, 4097, 8191, 8192, 8193, 16383,
              16384, 16385, 32769, 65535, 65536, 65537, 100003, (1 << 18) + 3, (1 << 20) - 1]


@pytest.mark.parametrize("ascending", [True, False])
def test_edge_sizes(ascending):
    for n in EDGE_SIZES:
        check_keys(workloads.uniform_u32(n, seed=n + 11), ascending)


@pytest.mark.parametrize("pad_front", [1, 2, 3])
def test_misaligned_pointers(pad_front):
    for n in [5, 4097, 16383, 16384, 70001, 1 << 18]:
        check_keys(workloads.uniform_u32(n, seed=n), True, pad_front)
        check_keys(workloads.uniform_u32(n, seed=n + 1), False, pad_front)


def test_pad_value_keys_and_all_equal():
    for n in [3, 1000, 16385, 1 << 17]:
        k = workloads.uniform_u32(n, seed=5)
        k[::3] = 0xFFFFFFFF
        k[1::5] = 0
        check_keys(k, True)
        check_keys(k, False)
        check_keys(np.full(n, 0xFFFFFFFF, dtype=np.uint32), True)
        check_keys(np.zeros(n, dtype=np.uint32), False)


def test_n16_uniform_workload():
    # single array of 2^16 uniform keys, ascending (the small configuration)
    check_keys(workloads.uniform_u32(1 << 16, seed=workloads.SEEDS["n16_uniform"]), True)


@pytest.mark.parametrize("dist", workloads.DISTRIBUTIONS)
def test_n24_distributions(dist):
    keys = workloads.keys_u32(dist, 1 << 24, seed=workloads.SEEDS["n24"])
    check_keys(keys, True)
    check_keys(keys, False)


def test_n24_non_power_of_two():
    keys = workloads.uniform_u32(10_000_019, seed=workloads.SEEDS["n24_npow2"])
    check_keys(keys, True)
    check_keys(keys, False)


@pytest.mark.parametrize("variant,tile,kpt,pipeline", [(1, 0, 0, 0), (2, 0, 0, 0), (0, 13, 0, 0), (0, 14, 5, 0),
                                                      (0, 14, 6, 1), (0, 13, 5, 1), (0, 14, 6, 2), (0, 13, 5, 2),
                                                      (0, 14, 6, 3)])
def test_variants_agree(variant, tile, kpt, pipeline):
    uncapped = pipeline == 3  # (pipeline column 3: the uncapped two-CTA kernel, one CTA per tile)
    bt.set_options(variant=variant, tile_log2=tile, keys_per_thread_log2=kpt, pipeline=0 if uncapped else pipeline,
                   l2_prefetch=0 if variant == 0 and tile == 13 else 1, ctas_per_sm=2 if uncapped else 3,
                   min_row_log2=3 if (kpt == 5 and pipeline == 0) else 0)
    for n in [3, 4097, 65537, 1 << 19]:
        check_keys(workloads.uniform_u32(n, seed=n), True)
        check_keys(workloads.uniform_u32(n, seed=n), False, 1)


def test_without_graphs_and_on_a_side_stream():
    bt.set_options(use_graph=0)
    check_keys(workloads.uniform_u32(300_000, seed=1), True)
    bt.set_options(use_graph=1)
    s = torch.cuda.Stream()
    keys = workloads.uniform_u32(300_001, seed=2)
    t = to_dev(keys)
    with torch.cuda.stream(s):
        bt.sort_(t)
    s.synchronize()
    assert np.array_equal(to_host(t), oracle.merge_sort(keys))
    # replaying the cached graph on the same buffer
    t.copy_(to_dev(keys))
    bt.sort_(t)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(t), oracle.merge_sort(keys))


def test_inside_user_graph_capture():
    keys = workloads.uniform_u32(200_000, seed=9)
    src = to_dev(keys)
    t = torch.empty_like(src)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        t.copy_(src)
        bt.sort_(t)  # warm-up outside capture builds plan state
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        t.copy_(src)
        bt.sort_(t)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(to_host(t), oracle.merge_sort(keys))


def test_profiled_launch_sequence():
    n = 1 << 20
    info = bt.plan_info(n)
    events = [torch.cuda.Event(enable_timing=True) for _ in range(info["launches"] + 1)]
    keys = workloads.uniform_u32(n, seed=4)
    t = to_dev(keys)
    kinds = bt.sort_profiled_(t, events)
    torch.cuda.synchronize()
    assert kinds[: info["launches"]][0] == 0
    assert np.array_equal(to_host(t), oracle.merge_sort(keys))
    times = [events[i].elapsed_time(events[i + 1]) for i in range(info["launches"])]
    assert all(x >= 0 for x in times)


@pytest.mark.parametrize("ascending,cap", [(True, 0), (False, 0), (True, 3)])
def test_pairs_small(ascending, cap):
    # cap 3: the composite tile kernel capped for three resident CTAs per SM
    bt.set_options(ctas_per_sm=cap)
    for n in [2, 3, 100, 4097, 8193, 70001, 1 << 18]:
        keys = (workloads.uniform_u32(n, seed=n) >> np.uint32(26)).astype(np.uint32)  # many ties
        vals = workloads.uniform_u32(n, seed=n + 7)
        tk, tv = to_dev(keys), to_dev(vals, 1)
        bt.sort_pairs_(tk, tv, ascending)
        torch.cuda.synchronize()
        wk, wv = oracle.merge_sort_pairs(keys, vals, ascending)
        assert np.array_equal(to_host(tk), wk) and np.array_equal(to_host(tv), wv), n


@pytest.mark.parametrize("ascending", [True, False])
def test_pairs_alignments_and_variants(ascending):
    # The optimized plan builds the composites in its first tile launch and
    # splits them in its last (vector accesses when the keys are 8-byte
    # aligned, element accesses otherwise; one launch does both up to 8192
    # pairs), then gathers the values by index; the basic and semi variants
    # use separate pack, gather and split kernels.  Keys equal to 0xFFFFFFFF
    # must still sort before the padding.
    for n in [5, 8191, 8192, 8193, 16385, (1 << 20) + 1]:
        keys = (workloads.uniform_u32(n, seed=n + 3) >> np.uint32(24)).astype(np.uint32)
        keys[::7] = 0xFFFFFFFF
        vals = workloads.uniform_u32(n, seed=n + 9)
        wk, wv = oracle.merge_sort_pairs(keys, vals, ascending)
        for kf, vf, variant in ((0, 0, 0), (1, 1, 0), (2, 0, 0), (0, 3, 0), (0, 0, 2), (1, 2, 1)):
            if variant == 1 and n > (1 << 14):
                continue
            bt.set_options(variant=variant)
            tk, tv = to_dev(keys, kf), to_dev(vals, vf)
            bt.sort_pairs_(tk, tv, ascending)
            torch.cuda.synchronize()
            assert np.array_equal(to_host(tk), wk) and np.array_equal(to_host(tv), wv), (n, kf, vf, variant)
    bt.set_options(variant=0)


def test_bounded_wait_times_out_and_context_stays_usable():
    # The pipelined kernels' mbarrier waits are bounded.  In the test mode
    # each CTA arms its barrier for its first tile's bulk copies but issues
    # none, so with a bound of 8 tries its wait runs out with no copy in
    # flight: the kernel writes BITONIC_ERR_TIMEOUT to the device status word
    # and returns.  A normal sort on the same context afterwards is exact.
    keys = workloads.uniform_u32(1 << 20, seed=19)
    bt.set_options(pipeline=1, use_graph=0)
    try:
        bt.debug_set_wait(True, 8)
        t = to_dev(keys)
        bt.sort_(t)
        assert bt.last_device_error() == bt.ERR_TIMEOUT
    finally:
        bt.debug_set_wait(False)
    assert bt.last_device_error() == bt.OK
    for pipeline in (1, 0):
        bt.set_options(pipeline=pipeline, use_graph=1)
        t = to_dev(keys)
        bt.sort_(t)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(t), oracle.merge_sort(keys)), pipeline


def test_pairs_n26_ties_by_index():
    # 2^26 pairs: keys uniform over [0, 2^20), values = original index
    keys, vals = workloads.pair_keys_u32(1 << 26, seed=workloads.SEEDS["pairs_n26"])
    tk, tv = to_dev(keys), to_dev(vals)
    bt.sort_pairs_(tk, tv, True)
    torch.cuda.synchronize()
    gk, gv = to_host(tk), to_host(tv)
    wk, wv = oracle.merge_sort_pairs(keys, vals, True)
    assert np.array_equal(gk, wk) and np.array_equal(gv, wv)



@pytest.mark.parametrize("n, kf, vf, ascending", [((1 << 24) + 5, 0, 0, True), (3 * (1 << 23) + 3, 1, 2, False)])
def test_pairs_sliced_gather_ragged(n, kf, vf, ascending):
    # Above 2^24 pairs the values are gathered in slices of at most 2^24
    # sources, one launch per slice (two here), each launch's ragged tail
    # handled element by element; keys and values off 16-byte boundaries in
    # the second case.
    keys = (workloads.uniform_u32(n, seed=n + 11) >> np.uint32(12)).astype(np.uint32)
    vals = workloads.uniform_u32(n, seed=n + 13)
    wk, wv = oracle.merge_sort_pairs(keys, vals, ascending)
    tk, tv = to_dev(keys, kf), to_dev(vals, vf)
    bt.sort_pairs_(tk, tv, ascending)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(tk), wk) and np.array_equal(to_host(tv), wv)
    assert bt.plan_info(n, pairs=True)["launches"] == bt.plan_info(n, pairs=True)["hbm_passes"] + 2

def segments_case(lens, seed, gap_every=0):
    lens = np.asarray(lens, dtype=np.int64)
    offs = np.zeros(lens.size + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    offs += 3  # offsets[0] need not be 0; starts land off 16-byte boundaries
    keys = workloads.uniform_u32(int(offs[-1]), seed)
    return keys, offs.astype(np.int32)


def check_segmented(keys, offs, pairs=False):
    tk = to_dev(keys)
    to = torch.from_numpy(offs).cuda()
    if pairs:
        vals = workloads.uniform_u32(keys.size, seed=77)
        tv = to_dev(vals)
        bt.sort_segmented_pairs_(tk, tv, to)
        torch.cuda.synchronize()
        wk, wv = oracle.segmented_sort_pairs(keys, vals, offs)
        assert np.array_equal(to_host(tk), wk) and np.array_equal(to_host(tv), wv)
    else:
        bt.sort_segmented_(tk, to)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(tk), oracle.segmented_sort(keys, offs))


@pytest.mark.parametrize("pairs", [False, True])
def test_segmented_edge_cases(pairs):
    lens = [0, 1, 2, 3, 0, 31, 32, 33, 4095, 4096, 4097, 8191, 8192, 8193, 16383, 16384, 16385,
            40000, 0, 1, 5]
    keys, offs = segments_case(lens, seed=12)
    check_segmented(keys, offs, pairs)


def check_segmented_descending(keys, offs, pairs):
    # expected: every segment sorted descending by the oracle (pairs: equal
    # keys in ascending original index); keys outside the span untouched
    tk = to_dev(keys)
    to = torch.from_numpy(offs).cuda()
    wk = keys.copy()
    if pairs:
        vals = workloads.uniform_u32(keys.size, seed=78)
        tv = to_dev(vals)
        bt.sort_segmented_pairs_(tk, tv, to, ascending=False)
        wv = vals.copy()
        for a, b in zip(offs[:-1], offs[1:]):
            if b > a:
                wk[a:b], wv[a:b] = oracle.merge_sort_pairs(keys[a:b], vals[a:b], False)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(tk), wk) and np.array_equal(to_host(tv), wv)
    else:
        bt.sort_segmented_(tk, to, ascending=False)
        for a, b in zip(offs[:-1], offs[1:]):
            if b > a:
                wk[a:b] = oracle.merge_sort(keys[a:b], False)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(tk), wk)


@pytest.mark.parametrize("pairs", [False, True])
def test_segmented_descending(pairs):
    # edge lengths (empty, single, tile boundaries, longer than a tile) after
    # 3 leading keys that lie outside every segment, then a mixed batch
    lens = [0, 1, 2, 3, 0, 31, 32, 33, 4095, 4096, 4097, 8191, 8192, 8193, 16384, 16385, 40000, 0, 1, 5]
    keys, offs = segments_case(lens, seed=13)
    keys[:3] = np.uint32(0xFFFFFFFF)
    check_segmented_descending(keys, offs, pairs)
    keys, offs = workloads.segmented_u32(3000, seed=6, max_len=20000)
    if pairs:  # many ties, so that the index order of equal keys is tested
        keys = (keys >> np.uint32(24)).astype(np.uint32)
    check_segmented_descending(keys, offs, pairs)


@pytest.mark.parametrize("pad_front", [0, 1, 3])
def test_segmented_long_segments(pad_front):
    # Segments longer than one tile run the multi-pass plan of a 2^k-key sort
    # (one persistent launch for all of them); among them 2^15, 2^17 and 2^20
    # keys, lengths just past a tile and ragged ones, between small segments,
    # with the keys array itself off a 16-byte boundary by pad_front keys.
    lens = [5, 1 << 15, 0, 1 << 17, 100, 1 << 20, 16385, (1 << 15) + 3, 3, 40000, (1 << 18) - 1, 8192, 1,
            (1 << 16) + 1, 2]
    keys, offs = segments_case(lens, seed=31 + pad_front)
    keys[::11] = keys[7]  # repeated keys
    tk = to_dev(keys, pad_front)
    to = torch.from_numpy(offs).cuda()
    want = oracle.segmented_sort(keys, offs)
    for _ in range(2):  # the second call reuses the workspace and the cached graph
        tk.copy_(to_dev(keys, pad_front))
        bt.sort_segmented_(tk, to)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(tk), want)
    assert bt.last_device_error() == bt.OK
    # descending: every segment reversed order, keys outside the segments untouched
    tk = to_dev(keys, pad_front)
    bt.sort_segmented_(tk, to, ascending=False)
    wk = keys.copy()
    for a, b in zip(offs[:-1], offs[1:]):
        if b > a:
            wk[a:b] = want[a:b][::-1]
    torch.cuda.synchronize()
    assert np.array_equal(to_host(tk), wk)


@pytest.mark.parametrize("pad_front", [0, 1])
def test_segmented_pairs_long_segments(pad_front):
    # Pair segments longer than one 8K-composite tile run the multi-pass plan
    # of a 2^k composite sort in the persistent launch, with pack, gather and
    # split passes; many ties, so that equal keys must keep their index order.
    lens = [3, 1 << 15, 8193, 0, 1 << 17, 100, (1 << 20) + 7, 8192, 40000, 1, (1 << 16) - 1]
    keys, offs = segments_case(lens, seed=51 + pad_front)
    keys = (keys >> np.uint32(22)).astype(np.uint32)
    vals = workloads.uniform_u32(keys.size, seed=52)
    wk, wv = oracle.segmented_sort_pairs(keys, vals, offs)
    to = torch.from_numpy(offs).cuda()
    for _ in range(2):
        tk, tv = to_dev(keys, pad_front), to_dev(vals, 1 - pad_front)
        bt.sort_segmented_pairs_(tk, tv, to)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(tk), wk) and np.array_equal(to_host(tv), wv)
    assert bt.last_device_error() == bt.OK
    # descending: by key descending, equal keys in ascending index
    tk, tv = to_dev(keys, pad_front), to_dev(vals, 1 - pad_front)
    bt.sort_segmented_pairs_(tk, tv, to, ascending=False)
    dk, dv = keys.copy(), vals.copy()
    for a, b in zip(offs[:-1], offs[1:]):
        if b > a:
            dk[a:b], dv[a:b] = oracle.merge_sort_pairs(keys[a:b], vals[a:b], False)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(tk), dk) and np.array_equal(to_host(tv), dv)


def test_segmented_many_long_segments():
    # 300 segments of 16385..70000 keys (a few passes each, many segments per
    # size class) and one of 2^21: the work of every pass interleaves segments
    rng = np.random.default_rng(4)
    lens = rng.integers(16385, 70001, size=300).tolist() + [1 << 21]
    keys, offs = segments_case(lens, seed=41)
    tk = to_dev(keys)
    bt.sort_segmented_(tk, torch.from_numpy(offs).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(to_host(tk), oracle.segmented_sort(keys, offs))
    # the same batch as pairs
    keys = (keys >> np.uint32(20)).astype(np.uint32)
    vals = np.arange(keys.size, dtype=np.uint32)
    tk, tv = to_dev(keys), to_dev(vals)
    bt.sort_segmented_pairs_(tk, tv, torch.from_numpy(offs).cuda())
    torch.cuda.synchronize()
    wk, wv = oracle.segmented_sort_pairs(keys, vals, offs)
    assert np.array_equal(to_host(tk), wk) and np.array_equal(to_host(tv), wv)


def test_segmented_batched_workload():
    # 65,536 arrays, lengths log-uniform in [1, 8192]
    keys, offs = workloads.segmented_u32(65536, seed=workloads.SEEDS["segmented"])
    check_segmented(keys, offs)


def test_segmented_pairs_mixed():
    keys, offs = workloads.segmented_u32(3000, seed=5, max_len=20000)
    check_segmented(keys, offs, pairs=True)


@pytest.mark.parametrize("seed", [28])
def test_n28_uniform_full(seed):
    # 2^28 uniform keys (1 GiB), the headline size
    keys = workloads.uniform_u32(1 << 28, seed=workloads.SEEDS["n28_uniform"])
    t = to_dev(keys)
    bt.sort_(t, True)
    torch.cuda.synchronize()
    got = to_host(t)
    del t
    torch.cuda.empty_cache()
    want = oracle.merge_sort(keys, True)
    assert np.array_equal(got, want)


def test_segmented_pairs_bounded_is_asynchronous_path():
    keys, offs = workloads.segmented_u32(5000, seed=8, max_len=8192)
    vals = workloads.uniform_u32(keys.size, seed=81)
    tk, tv = to_dev(keys), to_dev(vals)
    to = torch.from_numpy(offs).cuda()
    bt.sort_segmented_pairs_bounded_(tk, tv, to, 8192)
    torch.cuda.synchronize()
    wk, wv = oracle.segmented_sort_pairs(keys, vals, offs)
    assert np.array_equal(to_host(tk), wk) and np.array_equal(to_host(tv), wv)


def test_segmented_many_tiny_and_class_boundaries():
    # every class boundary 2^k and 2^k + 1, plus many length-2..16 segments
    lens = []
    for k in range(1, 15):
        lens += [1 << k, (1 << k) + 1, (1 << k) - 1]
    lens += [2, 3, 5, 9, 16, 17] * 500
    keys, offs = segments_case(lens, seed=21)
    check_segmented(keys, offs)
    keys2, offs2 = segments_case([l for l in lens if l <= 8192], seed=22)
    check_segmented(keys2, offs2, pairs=True)


TYPED_TORCH = {"int32": "int32", "float32": "float32", "uint64": "int64", "int64": "int64", "float64": "float64"}


def to_dev_typed(a: np.ndarray, pad_front: int = 0):
    """numpy keys -> CUDA tensor with the same bits, starting pad_front keys
    past an allocation boundary (so 4- and 8-byte keys can sit off a 16-byte
    boundary)."""
    dt = getattr(torch, TYPED_TORCH[a.dtype.name])
    raw = np.zeros(a.size + pad_front, dtype=a.dtype)
    raw[pad_front:] = a
    host = torch.from_numpy(raw.view(np.int64 if a.dtype.itemsize == 8 else np.int32)).view(dt)
    return host.cuda()[pad_front:]


def typed_host(t, like: np.ndarray) -> np.ndarray:
    return t.cpu().view(torch.int64 if like.dtype.itemsize == 8 else torch.int32).numpy().view(like.dtype)


def check_typed(keys, ascending, pad_front=0):
    t = to_dev_typed(keys, pad_front)
    bt.sort_typed_(t, ascending, key_type=keys.dtype.name)
    torch.cuda.synchronize()
    got = typed_host(t, keys)
    want = oracle.bitonic_sort_typed(keys, ascending)[0]
    ubits = np.uint64 if keys.dtype.itemsize == 8 else np.uint32
    assert np.array_equal(got.view(ubits), want.view(ubits)), (keys.dtype.name, keys.size, ascending, pad_front)


@pytest.mark.parametrize("kind", workloads.TYPED_KEY_KINDS)
@pytest.mark.parametrize("ascending", [True, False])
def test_typed_keys_against_oracle(kind, ascending):
    # Special values everywhere (signed zeros, infinities, NaNs of both signs
    # and kinds, subnormals, integer extremes); sizes over several tiles with
    # ragged tails, and a pointer off the 16-byte boundary.
    for n in [2, 3, 7, 1000, 8193, 65537, (1 << 18) + 5]:
        keys = workloads.typed_keys(kind, n, seed=n)
        check_typed(keys, ascending)
    check_typed(workloads.typed_keys(kind, 70001, seed=4), ascending, pad_front=1)


@pytest.mark.parametrize("kind", workloads.TYPED_KEY_KINDS)
def test_typed_keys_large_against_library_sort(kind):
    # 2^24 keys (several global passes) without NaNs or -0, where numpy's
    # order is the type's total order.
    keys = workloads.typed_keys(kind, 1 << 24, seed=24, specials=False)
    want = np.sort(keys)
    ubits = np.uint64 if keys.dtype.itemsize == 8 else np.uint32
    for asc in (True, False):
        t = to_dev_typed(keys)
        bt.sort_typed_(t, asc, key_type=kind)
        torch.cuda.synchronize()
        got = typed_host(t, keys)
        assert np.array_equal(got.view(ubits), (want if asc else want[::-1]).view(ubits)), (kind, asc)


@pytest.mark.parametrize("kind", workloads.TYPED_KEY_KINDS)
def test_typed_keys_multi_pass_against_oracle(kind):
    # 2^21 + 5 keys (global passes and a ragged tail) with the special values
    # mixed in (NaNs of both signs and kinds, signed zeros, infinities,
    # subnormals, integer extremes), against the typed oracle.  Distinct bit
    # patterns are distinct in the type's total order, so the descending
    # result is exactly the ascending one reversed.
    keys = workloads.typed_keys(kind, (1 << 21) + 5, seed=21, specials=True)
    want, _ = oracle.bitonic_sort_typed(keys, True)
    ubits = np.uint64 if keys.dtype.itemsize == 8 else np.uint32
    for asc in (True, False):
        t = to_dev_typed(keys)
        bt.sort_typed_(t, asc, key_type=kind)
        torch.cuda.synchronize()
        got = typed_host(t, keys)
        assert np.array_equal(got.view(ubits), (want if asc else want[::-1]).view(ubits)), (kind, asc)


@pytest.mark.parametrize("variant,pipeline", [(1, 0), (2, 0), (0, 1)])
@pytest.mark.parametrize("kind", ["float32", "int32", "float64", "int64"])
def test_typed_keys_other_variants(kind, variant, pipeline):
    # The basic variant's one-step kernels and the pipelined kernels take the
    # key map as separate passes (floats) or as XOR masks (signed integers).
    bt.set_options(variant=variant, pipeline=pipeline)
    for n in [5, 4097, 65537]:
        keys = workloads.typed_keys(kind, n, seed=n + 11)
        check_typed(keys, True)
        check_typed(keys, False)


def host_tensor(a: np.ndarray, pinned=True):
    t = torch.from_numpy(a.view(np.int32).copy())
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("ascending", [True, False])
def test_host_buffer_sort(ascending):
    # Sizes: one tile (a single launch), a partial last chunk, several
    # chunks of a multi-pass plan, and 2^22 keys.
    for n in [1, 2, 1000, 16384, 16385, 100003, (1 << 20) + 3, 1 << 22]:
        keys = workloads.uniform_u32(n, seed=n + 5)
        src, dst = host_tensor(keys), host_tensor(np.zeros(n, np.uint32))
        bt.sort_host(src, dst, ascending)
        torch.cuda.synchronize()
        assert np.array_equal(dst.numpy().view(np.uint32), oracle.merge_sort(keys, ascending)), n
        assert np.array_equal(src.numpy().view(np.uint32), keys)   # the input is left alone


def test_host_buffer_sort_in_place_pageable_and_basic_variant():
    keys = workloads.uniform_u32(300_001, seed=8)
    t = host_tensor(keys)
    bt.sort_host(t)                                  # in == out
    torch.cuda.synchronize()
    assert np.array_equal(t.numpy().view(np.uint32), oracle.merge_sort(keys))
    p = host_tensor(keys, pinned=False)              # pageable memory
    bt.sort_host(p, ascending=False)
    torch.cuda.synchronize()
    assert np.array_equal(p.numpy().view(np.uint32), oracle.merge_sort(keys, False))
    bt.set_options(variant=1)                        # one-step kernels: upload, sort, download in turn
    q = host_tensor(keys[:5000])
    bt.sort_host(q)
    torch.cuda.synchronize()
    assert np.array_equal(q.numpy().view(np.uint32), oracle.merge_sort(keys[:5000]))


def test_host_buffer_sorts_on_two_streams_overlap_correctly():
    # Two calls in flight on different streams, each with its own device buffer.
    a_keys, b_keys = workloads.uniform_u32(1 << 21, seed=1), workloads.uniform_u32((1 << 21) - 7, seed=2)
    a_in, b_in = host_tensor(a_keys), host_tensor(b_keys)
    a_out, b_out = host_tensor(np.zeros_like(a_keys)), host_tensor(np.zeros_like(b_keys))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(2):
        bt.sort_host(a_in, a_out, True, stream=s1)
        bt.sort_host(b_in, b_out, False, stream=s2)
    torch.cuda.synchronize()
    assert np.array_equal(a_out.numpy().view(np.uint32), oracle.merge_sort(a_keys))
    assert np.array_equal(b_out.numpy().view(np.uint32), oracle.merge_sort(b_keys, False))


@pytest.mark.parametrize("ascending", [True, False])
def test_host_buffer_batch(ascending):
    # Mixed sizes (empty, one key, one tile, several chunks), in place and
    # not, and an output buffer reused by arrays two apart (the later wins).
    sizes = [0, 1, 5, 16384, 100003, (1 << 20) + 7, 1 << 21, 3000]
    keys = [workloads.uniform_u32(n, seed=100 + i) for i, n in enumerate(sizes)]
    ins = [host_tensor(k) for k in keys]
    outs = [host_tensor(np.zeros(n, np.uint32)) if i % 3 else ins[i] for i, n in enumerate(sizes)]
    bt.sort_host_batch(ins, outs, ascending)
    torch.cuda.synchronize()
    for i, k in enumerate(keys):
        assert np.array_equal(outs[i].numpy().view(np.uint32), oracle.merge_sort(k, ascending)), sizes[i]
    # the same call again: the arrays between the first and the last replay
    # the device-sort graphs captured the first time (one per device buffer)
    ins = [host_tensor(k) for k in keys]
    outs = [host_tensor(np.zeros(n, np.uint32)) for n in sizes]
    bt.sort_host_batch(ins, outs, ascending)
    torch.cuda.synchronize()
    for i, k in enumerate(keys):
        assert np.array_equal(outs[i].numpy().view(np.uint32), oracle.merge_sort(k, ascending)), sizes[i]
    shared = host_tensor(np.zeros(1 << 20, np.uint32))
    a, b = workloads.uniform_u32(1 << 20, seed=7), workloads.uniform_u32(1 << 20, seed=8)
    bt.sort_host_batch([host_tensor(a), host_tensor(np.zeros(3, np.uint32)), host_tensor(b)],
                       [shared, host_tensor(np.zeros(3, np.uint32)), shared], ascending)
    torch.cuda.synchronize()
    assert np.array_equal(shared.numpy().view(np.uint32), oracle.merge_sort(b, ascending))


def unsigned_signature(t, chunk=1 << 27):
    """Multiset signature of a CUDA int32 tensor read as uint32: the 4096-bucket
    histogram of the top 12 bits, and the sums of the keys and of their
    squares (modulo 2^64)."""
    hist = torch.zeros(4096, dtype=torch.int64, device=t.device)
    s1 = torch.zeros((), dtype=torch.int64, device=t.device)
    s2 = torch.zeros((), dtype=torch.int64, device=t.device)
    for c in range(0, t.numel(), chunk):
        x = t[c:c + chunk].to(torch.int64) & 0xFFFFFFFF
        hist += torch.bincount(x >> 20, minlength=4096)
        s1 += x.sum()
        s2 += (x * x).sum()
    return hist, int(s1), int(s2)


def assert_sorted_unsigned(t, chunk=1 << 27):
    flip = torch.tensor(-2 ** 31, dtype=torch.int32, device=t.device)
    prev = None
    for c in range(0, t.numel(), chunk):
        u = torch.bitwise_xor(t[c:c + chunk], flip)   # unsigned order as signed order
        assert bool((u[1:] >= u[:-1]).all()), c
        if prev is not None:
            assert int(u[0]) >= prev, c
        prev = int(u[-1])


def test_maximum_size_properties():
    # The largest supported sort, 2^31 keys (8 GiB), and 2^31 - 5 (a ragged
    # tail at the limit): too large for the oracle, so checked by properties
    # that hold at any size -- sorted, the same multiset signature as the
    # input, and the extremes in place.  Input: a seeded device generator.
    n = 1 << 31
    gen = torch.Generator(device="cuda").manual_seed(31)
    src = torch.randint(-2 ** 31, 2 ** 31, (n,), dtype=torch.int32, device="cuda", generator=gen)
    for m in (n, n - 5):
        t = src[:m].clone()
        bt.sort_(t)
        torch.cuda.synchronize()
        assert_sorted_unsigned(t)
        h_in, a_in, b_in = unsigned_signature(src[:m])
        h_out, a_out, b_out = unsigned_signature(t)
        assert torch.equal(h_in, h_out) and a_in == a_out and b_in == b_out, m
        flipped = torch.bitwise_xor(src[:m], torch.tensor(-2 ** 31, dtype=torch.int32, device="cuda"))
        lo, hi = int(flipped.min()) + 2 ** 31, int(flipped.max()) + 2 ** 31
        assert int(t[0]) & 0xFFFFFFFF == lo and int(t[-1]) & 0xFFFFFFFF == hi, m
        del t, flipped
    del src
    torch.cuda.empty_cache()


@pytest.mark.parametrize("split,graphs", [(1, 1), (2, 1), (1, 0), (2, 0)])
def test_split_tile_ranges_agree_with_oracle(split, graphs):
    # The leading launches of a graph-captured sort as 2 or 4 concurrent
    # tile ranges: sizes with several global passes, a ragged tail with
    # tiles past the last key, an off-boundary front, both directions; pairs
    # (whose first and last launches stay whole) and 8-byte keys; and a sort
    # captured inside a caller's graph (which stays unsplit), followed by a
    # split sort on another stream while that graph still exists.
    # graphs = 0: plain launches, split in two on a second stream of the
    # caller's stream's own
    bt.set_options(split_log2=split, use_graph=graphs)
    for n in [1 << 16, (1 << 20) + 3, 1 << 22, 10_000_019]:
        keys = workloads.uniform_u32(n, seed=n + 5)
        check_keys(keys, True)
        check_keys(keys, False, 1)
    n = (1 << 21) + 5
    keys = (workloads.uniform_u32(n, seed=3) >> np.uint32(20)).astype(np.uint32)
    vals = workloads.uniform_u32(n, seed=4)
    wk, wv = oracle.merge_sort_pairs(keys, vals, False)
    tk, tv = to_dev(keys), to_dev(vals)
    bt.sort_pairs_(tk, tv, False)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(tk), wk) and np.array_equal(to_host(tv), wv)
    k64 = workloads.typed_keys("uint64", (1 << 20) + 7, seed=5, specials=True)
    check_typed(k64, True)
    check_typed(k64, False, 1)
    keys = workloads.uniform_u32((1 << 20) + 3, seed=6)
    src = to_dev(keys)
    t = torch.empty_like(src)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        t.copy_(src)
        bt.sort_(t)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        t.copy_(src)
        bt.sort_(t)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(to_host(t), oracle.merge_sort(keys))
    other = workloads.uniform_u32(1 << 22, seed=8)
    t2 = to_dev(other)
    s2 = torch.cuda.Stream()
    with torch.cuda.stream(s2):
        bt.sort_(t2)
    s2.synchronize()
    assert np.array_equal(to_host(t2), oracle.merge_sort(other))
