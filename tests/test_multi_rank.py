"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Queries are independent per seed, so ranks are replicas that split the seed
stream; the only cross-rank steps are a barrier and the max of the step time.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    all_seeds = np.arange(10 * w, dtype=np.int32)
    mine = bench.shard_seeds(all_seeds, r, w, 10)
    bench.barrier(w)
    t = bench.max_over_ranks(1.0 + r, w)
    q.put((r, mine.tolist(), t))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in range(2))
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (r0, s0, t0), (r1, s1, t1) = res
    assert set(s0).isdisjoint(s1) and sorted(s0 + s1) == list(range(20))
    assert t0 == t1 == 2.0
