"""The multi-GPU bench path on CPU: world_size-2 gloo ranks (replicas, no
data-path collective; only the job time is reduced, by max over ranks)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import workloads
    slowest = bench.reduce_max(10.0 + 5.0 * rank, world)
    seed = bench.replica_seed(rank)
    keys = workloads.uniform_u32(1000, seed=seed)
    q.put((rank, slowest, seed, int(keys[:8].sum())))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_and_own_inputs():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    assert res[0][1] == res[1][1] == 15.0            # max over ranks
    assert res[0][2] != res[1][2] and res[0][3] != res[1][3]   # each rank sorts its own array
