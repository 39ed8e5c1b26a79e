"""Two ranks, two library instances, disjoint seed shards (one GPU).

Queries are independent per seed, so bench.py's ranks are replicas that split
one global seed stream (`shard_seeds`) and meet only at a barrier and the max
of the step time.  Here two spawned processes each load the library, build the
same graph, preprocess it and answer their shard; rank 0 gathers the shards
over gloo.  The union must match a one-rank run of the whole stream column by
column, and sampled columns must match the FP64 oracle.  The ranks share the
GPU by time-slicing; their kernels never wait on one another (the only
cross-rank steps are host-side gloo calls).
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SCALE, EF, PER_RANK = 14, 16, 20
C, S, T, EPS = 0.15, 5, 10, 1e-9


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _scores(seeds):
    import torch
    import synth
    import paper_1708_02574_gb300 as tpa
    n = 1 << SCALE
    src, dst = synth.rmat_edges(SCALE, EF)
    g = tpa.build_graph(n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    tpa.preprocess(g, C, T, EPS)
    out = tpa.query(g, torch.from_numpy(seeds).cuda(), S).cpu().numpy()
    g.free()
    return out


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK="0")
    import torch
    import torch.distributed as dist
    import bench
    import synth
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    n = 1 << SCALE
    src, dst = synth.rmat_edges(SCALE, EF)
    all_seeds = synth.query_seeds(synth.nodes_with_out_edge(n, src, dst), PER_RANK * w)
    mine = bench.shard_seeds(all_seeds, r, w, PER_RANK)
    out = torch.from_numpy(np.ascontiguousarray(_scores(mine)))
    parts = [torch.empty_like(out) for _ in range(w)] if r == 0 else None
    dist.gather(out, parts, dst=0)
    bench.barrier(w)
    if r == 0:
        q.put((all_seeds, torch.cat(parts, dim=1).numpy()))
    dist.destroy_process_group()


@pytest.mark.timeout(600)
def test_two_ranks_union_equals_one_rank():
    import torch.multiprocessing as mp
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    all_seeds, union = q.get(timeout=540)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert union.shape == (1 << SCALE, 2 * PER_RANK)
    one = _scores(all_seeds)
    # the same seeds, chunked differently: per-column arithmetic may take the
    # push or the pull branch depending on a chunk's other seeds
    diff = np.abs(union.astype(np.float64) - one)
    assert diff.sum(axis=0).max() <= 1e-5 and diff.max() <= 1e-7
    n = 1 << SCALE
    src, dst = synth.rmat_edges(SCALE, EF)
    og = oracle.build_graph(n, src, dst)
    rs, _ = oracle.preprocess(og, C, T, EPS)
    for j in (0, PER_RANK - 1, PER_RANK, 2 * PER_RANK - 1):
        ref = oracle.query(og, int(all_seeds[j]), C, S, T, rs, EPS)
        d = np.abs(union[:, j].astype(np.float64) - ref)
        assert d.sum() <= 1e-5 and d.max() <= 1e-7, f"column {j}: L1 {d.sum():.3e} max {d.max():.3e}"
