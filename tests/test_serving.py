"""Serving loop: arena bookkeeping (CPU) and, on the GPU, that every request
of a mixed Poisson stream comes back exactly as the oracle sorts it, and
exactly as the library sorts it alone."""
import numpy as np
import pytest

import oracle
import workloads
from paper_1506_01446_gb300.serving import Arena


def test_arena_first_fit_and_coalescing():
    a = Arena(1 << 20)
    blocks = [a.alloc(1000 + 37 * i) for i in range(50)]
    assert all(b is not None for b in blocks)
    assert all(b[0] % 16 == 0 for b in blocks)
    offs = sorted(blocks)
    for (o1, l1), (o2, _) in zip(offs, offs[1:]):
        assert o1 + l1 <= o2                               # no overlap
    for b in blocks[::2]:
        a.release(b)
    for b in blocks[1::2]:
        a.release(b)
    assert a.free == [(0, 1 << 20)] and a.used == 0       # fully coalesced
    assert a.alloc(2 << 20) is None                         # larger than the budget


def _serve(n_req, seed, budget, hi_log2, rate=2000.0, engine="native"):
    torch = pytest.importorskip("torch")
    from paper_1506_01446_gb300.serving import SortServer
    arr, sizes, hv = workloads.serving_requests(n_req, seed=seed, rate=rate, lo_log2=10, hi_log2=hi_log2)
    pool = workloads.uniform_u32(1 << 23, seed=seed + 1)
    pool_v = workloads.uniform_u32(1 << 23, seed=seed + 2)
    srv = SortServer(pool, pool_v, budget_bytes=budget, streams=4)
    if budget >= 1 << 30:
        srv.warmup(int(sizes.max()))
    stats, outs = srv.run(arr, sizes, hv, keep_outputs=True, engine=engine)
    reqs = [(srv._kind(int(n), bool(h)), int(n), bool(h)) for n, h in zip(sizes, hv)]
    return srv, stats, outs, reqs, pool, pool_v, torch


@pytest.mark.gpu
@pytest.mark.parametrize("engine", ["native", "python"])
def test_mixed_stream_results_match_oracle_and_alone(engine):
    import paper_1506_01446_gb300 as bt
    srv, stats, outs, reqs, pool, pool_v, torch = _serve(300, 5, 1 << 30, hi_log2=17, engine=engine)
    assert stats["requests"] == 300 and stats["batches"] > 0
    # re-derive each request's input slice the way the server assigned it
    probe = type(srv).__new__(type(srv))
    probe.rings, probe.ring_pos = srv.rings, {k: 0 for k in srv.rings}
    for i, (kind, n, has_v) in enumerate(reqs):
        src = type(srv)._src(probe, kind, n)
        k_in, v_in = pool[src:src + n], pool_v[src:src + n]
        got_k, got_v = outs[i]
        if has_v:
            wk, wv = oracle.merge_sort_pairs(k_in, v_in)
            assert np.array_equal(got_k, wk) and np.array_equal(got_v, wv), i
            tk = torch.from_numpy(k_in.view(np.int32).copy()).cuda()
            tv = torch.from_numpy(v_in.view(np.int32).copy()).cuda()
            bt.sort_pairs_(tk, tv)                            # the same request alone
            assert np.array_equal(tk.cpu().numpy().view(np.uint32), got_k)
            assert np.array_equal(tv.cpu().numpy().view(np.uint32), got_v)
        else:
            assert np.array_equal(got_k, oracle.merge_sort(k_in)), i
            tk = torch.from_numpy(k_in.view(np.int32).copy()).cuda()
            bt.sort_(tk)
            assert np.array_equal(tk.cpu().numpy().view(np.uint32), got_k)


@pytest.mark.gpu
@pytest.mark.parametrize("engine", ["native", "python"])
def test_tiny_budget_still_serves_everything(engine):
    srv, stats, outs, reqs, pool, pool_v, torch = _serve(80, 9, 6 << 20, hi_log2=18, engine=engine)
    assert stats["peak_device_bytes"] <= 6 << 20
    assert all(o is not None for o in outs)
    for (k, v), (_, n, has_v) in zip(outs, reqs):
        assert k.size == n and np.all(k[1:] >= k[:-1])


@pytest.mark.gpu
@pytest.mark.parametrize("engine", ["native", "python"])
def test_batched_stream_packs_many_requests_and_matches_oracle(engine):
    # A stream fast enough that requests overlap (200,000 req/s, sizes up to
    # 2^14 keys): the loop packs many requests into each segmented launch,
    # and every result is still exactly the oracle's and the same as the
    # request sorted alone.
    import paper_1506_01446_gb300 as bt
    srv, stats, outs, reqs, pool, pool_v, torch = _serve(600, 7, 1 << 30, hi_log2=14, rate=200000.0, engine=engine)
    assert stats["mean_batch"] > 4, stats
    probe = type(srv).__new__(type(srv))
    probe.rings, probe.ring_pos = srv.rings, {k: 0 for k in srv.rings}
    for i, (kind, n, has_v) in enumerate(reqs):
        src = type(srv)._src(probe, kind, n)
        k_in, v_in = pool[src:src + n], pool_v[src:src + n]
        got_k, got_v = outs[i]
        if has_v:
            wk, wv = oracle.merge_sort_pairs(k_in, v_in)
            assert np.array_equal(got_k, wk) and np.array_equal(got_v, wv), i
        else:
            assert np.array_equal(got_k, oracle.merge_sort(k_in)), i
        if i % 50 == 0:  # the same request alone
            tk = torch.from_numpy(k_in.view(np.int32).copy()).cuda()
            if has_v:
                tv = torch.from_numpy(v_in.view(np.int32).copy()).cuda()
                bt.sort_pairs_(tk, tv)
                assert np.array_equal(tv.cpu().numpy().view(np.uint32), got_v)
            else:
                bt.sort_(tk)
            assert np.array_equal(tk.cpu().numpy().view(np.uint32), got_k)


@pytest.mark.gpu
@pytest.mark.parametrize("engine", ["native", "python"])
def test_server_leaves_other_threads_graph_mode_alone(engine):
    # The server turns graph replay off for its own thread only: the
    # process-wide option is unchanged during and after a run.
    import paper_1506_01446_gb300 as bt
    before = bt.get_options()["use_graph"]
    _serve(40, 11, 1 << 28, hi_log2=15, engine=engine)
    assert bt.get_options()["use_graph"] == before


@pytest.mark.gpu
def test_native_loop_splits_groups_larger_than_the_budget():
    # 1 MiB of device memory and 200,000 req/s of requests up to 2^14 keys:
    # the requests that wait together form packed groups larger than the
    # whole budget, which the native loop splits until the head fits.  Every
    # result must still be the oracle's.
    srv, stats, outs, reqs, pool, pool_v, torch = _serve(300, 13, 1 << 20, hi_log2=14, rate=200000.0)
    assert stats["peak_device_bytes"] <= 1 << 20
    probe = type(srv).__new__(type(srv))
    probe.rings, probe.ring_pos = srv.rings, {k: 0 for k in srv.rings}
    for i, (kind, n, has_v) in enumerate(reqs):
        src = type(srv)._src(probe, kind, n)
        k_in, v_in = pool[src:src + n], pool_v[src:src + n]
        got_k, got_v = outs[i]
        if has_v:
            wk, wv = oracle.merge_sort_pairs(k_in, v_in)
            assert np.array_equal(got_k, wk) and np.array_equal(got_v, wv), i
        else:
            assert np.array_equal(got_k, oracle.merge_sort(k_in)), i
