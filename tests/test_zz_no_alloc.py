"""The key/value sort that allocates no device memory.

bitonic_sort_pairs_u32_noalloc serves callers that cannot let a library call
cudaMalloc: applications whose own memory manager owns all device memory,
and latency-critical paths that cannot afford cudaMalloc's implicit
synchronisation.  Its result must be exactly the oracle's pair sort (keys in
order, equal keys by original index, values with their keys) and the same as
the allocating bitonic_sort_pairs_u32.  The file sorts last so that a run
stopping at the first failure has already run every other test, and it
passes both alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1506_01446_gb300 as bt  # noqa: E402

MAX_PAIRS = 1 << 20


def dev_u32(a, pad_front=0):
    """uint32 numpy -> int32 CUDA view starting pad_front elements past a
    16-byte boundary."""
    buf = np.zeros(a.size + pad_front, dtype=np.uint32)
    buf[pad_front:] = a
    return torch.from_numpy(buf.view(np.int32)).cuda()[pad_front:]


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def run_noalloc(keys, vals, ascending, kf=0, vf=0):
    lib = bt.load()
    stream = torch.cuda.current_stream().cuda_stream
    nk, nv = dev_u32(keys, kf), dev_u32(vals, vf)
    rc = lib.bitonic_sort_pairs_u32_noalloc(nk.data_ptr(), nv.data_ptr(), keys.size, int(ascending), stream)
    assert rc == bt.OK, bt.status_string(rc)
    torch.cuda.synchronize()
    return host_u32(nk), host_u32(nv)


def test_no_alloc_pair_sort_matches_the_oracle_twice_in_a_row():
    # two calls in a row share the fixed array: the second must not see the
    # first's contents
    cases = [((1 << 20) - 3, True, 11), (70_001, False, 12)]
    for n, ascending, seed in cases:
        keys = (workloads.uniform_u32(n, seed=seed) >> np.uint32(20)).astype(np.uint32)  # many ties
        vals = workloads.uniform_u32(n, seed=seed + 1)
        gk, gv = run_noalloc(keys, vals, ascending)
        wk, wv = oracle.merge_sort_pairs(keys, vals, ascending)
        assert np.array_equal(gk, wk) and np.array_equal(gv, wv), (n, ascending)
        # and the same as the allocating sort
        ak, av = dev_u32(keys), dev_u32(vals)
        bt.sort_pairs_(ak, av, ascending)
        torch.cuda.synchronize()
        assert np.array_equal(host_u32(ak), gk) and np.array_equal(host_u32(av), gv)


def test_no_alloc_at_its_limit_with_misaligned_pointers():
    # exactly 2^20 pairs (the array's size) and one fewer, keys and values
    # starting off 16-byte boundaries, both directions
    for n, kf, vf, ascending in ((MAX_PAIRS, 1, 3, True), (MAX_PAIRS - 1, 3, 2, False), (MAX_PAIRS, 0, 0, False)):
        keys = (workloads.uniform_u32(n, seed=n + kf) >> np.uint32(22)).astype(np.uint32)
        keys[::9] = 0xFFFFFFFF
        vals = workloads.uniform_u32(n, seed=n + vf + 5)
        gk, gv = run_noalloc(keys, vals, ascending, kf, vf)
        wk, wv = oracle.merge_sort_pairs(keys, vals, ascending)
        assert np.array_equal(gk, wk) and np.array_equal(gv, wv), (n, kf, vf, ascending)


def test_no_alloc_rejects_sizes_beyond_its_array():
    lib = bt.load()
    t = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = lib.bitonic_sort_pairs_u32_noalloc(t.data_ptr(), t.data_ptr(), MAX_PAIRS + 1, 1, None)
    assert rc == bt.ERR_UNSUPPORTED
