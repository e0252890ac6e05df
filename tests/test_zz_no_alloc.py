"""The key/value sort that allocates no device memory.

bitonic_sort_pairs_u32_noalloc serves callers that cannot let a library call
cudaMalloc (work captured into CUDA graphs, programs whose own allocator owns
all device memory, latency-critical paths).  It must give exactly what the
allocating bitonic_sort_pairs_u32 gives.  The file sorts last so that a run
stopping at the first failure has already run every other test, and it
passes both alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1506_01446_gb300 as bt  # noqa: E402

MAX_PAIRS = 1 << 20


def dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_no_alloc_pair_sort_matches_the_allocating_sort_twice_in_a_row():
    lib = bt.load()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [((1 << 20) - 3, True, 11), (70_001, False, 12)]   # two calls in a row
    for n, ascending, seed in cases:
        keys = (workloads.uniform_u32(n, seed=seed) >> np.uint32(20)).astype(np.uint32)  # many ties
        vals = workloads.uniform_u32(n, seed=seed + 1)
        nk, nv = dev_u32(keys), dev_u32(vals)
        ak, av = dev_u32(keys), dev_u32(vals)
        rc = lib.bitonic_sort_pairs_u32_noalloc(nk.data_ptr(), nv.data_ptr(), n, int(ascending), stream)
        assert rc == bt.OK, bt.status_string(rc)
        bt.sort_pairs_(ak, av, ascending)
        torch.cuda.synchronize()
        # sorted keys/values have one correct answer: compare bit for bit
        assert np.array_equal(host_u32(nk), host_u32(ak))
        assert np.array_equal(host_u32(nv), host_u32(av))


def test_no_alloc_rejects_sizes_beyond_its_array():
    lib = bt.load()
    t = torch.zeros(16, dtype=torch.int32, device="cuda")
    rc = lib.bitonic_sort_pairs_u32_noalloc(t.data_ptr(), t.data_ptr(), MAX_PAIRS + 1, 1, None)
    assert rc == bt.ERR_UNSUPPORTED
