"""Batched serving with CUDA graphs (tpa_server) against tpa_query and the FP64 oracle.

R-MAT scale 14 (16,384 nodes, edge factor 16, key 1); request batches of
uneven size drawn uniformly from {1, 7, 32, 100, 256} (key 3) with seeds
uniform over nodes with an out-edge, the first batch of a size answered
directly and captured, later ones replayed.  The server orders the seeds of
a batch as tpa_query does (seeds of more than 256 out-edges into the last
chunks) and chooses the chunk branches on the host, so each batch must equal
tpa_query on the same seeds bit for bit; sampled columns must be within
L1 <= 1e-5 and max-abs <= 1e-7 of the oracle.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

C, S, T, EPS = 0.15, 5, 10, 1e-9


def tpa():
    import paper_1708_02574_gb300 as m
    return m


def parity(gpu, ref, tag):
    diff = np.abs(np.asarray(gpu, np.float64) - ref)
    assert diff.sum() <= 1e-5 and diff.max() <= 1e-7, f"{tag}: L1 {diff.sum():.3e} max {diff.max():.3e}"


def same_as_query(got, ref, seeds, outdeg, tag):
    """Bit for bit: the server runs the seeds in tpa_query's order with the
    same branches and kernels, and swaps the moved columns back the same way."""
    import torch
    assert torch.equal(got, ref), tag


@pytest.fixture(scope="module")
def graph14():
    n = 1 << 14
    s, d = synth.rmat_edges(14, 16)
    og = oracle.build_graph(n, s, d)
    g = tpa().build_graph(n, s, d)
    tpa().preprocess(g, C, T, EPS)
    rs, _ = oracle.preprocess(og, C, T, EPS)
    cand = synth.nodes_with_out_edge(n, s, d)
    return dict(n=n, og=og, g=g, rs=rs, cand=cand)


def test_server_uneven_batches(graph14):
    import torch
    t = tpa()
    sizes = synth.batch_sizes(1200)
    seeds_all = synth.query_seeds(graph14["cand"], sum(sizes), key=11)
    seeds_all[0] = 0                                  # a hub: its chunk takes the pull branch
    srv = t.Server(graph14["g"], S, max_k=256)
    off = 0
    for b, k in enumerate(sizes):
        sd = seeds_all[off:off + k]
        off += k
        got = srv.query(torch.from_numpy(sd).cuda() if b % 2 else sd).clone()
        ref = t.query(graph14["g"], sd, S)
        same_as_query(got, ref, sd, graph14["og"].outdeg, f"batch {b} (k={k}) differs from tpa_query")
        if b < 6:
            for j in sorted({0, k // 2, k - 1}):
                parity(got[:, j].cpu().numpy(),
                       oracle.query(graph14["og"], int(sd[j]), C, S, T, graph14["rs"], EPS), f"batch {b} col {j}")
    st = srv.stats(256)
    # every batch is a replay or a direct run + capture (graphs are keyed by
    # the batch size and the chunks' branches); a batch that grew the
    # workspace drops the graphs captured over the old buffers
    assert st["replays"] + st["captures"] == len(sizes)
    assert len(set(sizes)) <= st["captures"] and st["replays"] >= 1
    assert 1 <= st["graphs"] <= 64
    assert st["launches_per_replay"] > 0
    srv.sync()
    srv.free()


def test_server_workspace_growth_recaptures(graph14):
    """A batch of 1 seed runs chunks of width 1; a later batch of 256 needs
    chunks of 8 and grows every workspace buffer.  The graph captured for 1
    refers to the old buffers, so it must be dropped and captured again, not
    replayed."""
    import torch
    t = tpa()
    sd = synth.query_seeds(graph14["cand"], 256, key=14)
    srv = t.Server(graph14["g"], S, max_k=256)
    expect = [(1, dict(graphs=1, replays=0, captures=1)),
              (256, dict(graphs=1, replays=0, captures=2)),     # grew: the graph for 1 is gone
              (1, dict(graphs=2, replays=0, captures=3)),
              (1, dict(graphs=2, replays=1, captures=3)),
              (256, dict(graphs=2, replays=2, captures=3))]
    for k, st in expect:
        got = srv.query(sd[:k]).clone()
        same_as_query(got, t.query(graph14["g"], sd[:k], S), sd[:k], graph14["og"].outdeg, k)
        now = srv.stats(k)
        assert {key: now[key] for key in st} == st, (k, now)
    parity(got[:, 255].cpu().numpy(), oracle.query(graph14["og"], int(sd[255]), C, S, T, graph14["rs"], EPS), "k 256")
    srv.free()


def test_server_recaptures_after_setting_change(graph14):
    import torch
    t = tpa()
    seeds = synth.query_seeds(graph14["cand"], 32, key=12)
    srv = t.Server(graph14["g"], S, max_k=64)
    a = srv.query(seeds).clone()
    a2 = srv.query(seeds).clone()
    assert torch.equal(a, a2)
    try:
        t.set_batch_width(4)
        b = srv.query(seeds).clone()
        assert srv.stats()["graphs"] == 1            # the old graph was dropped, one new capture
        same_as_query(b, t.query(graph14["g"], seeds, S), seeds, graph14["og"].outdeg, "width 4")
        for j in (0, 31):
            parity(b[:, j].cpu().numpy(),
                   oracle.query(graph14["og"], int(seeds[j]), C, S, T, graph14["rs"], EPS), f"width 4 col {j}")
    finally:
        t.set_batch_width(0)
    srv.free()


@pytest.mark.parametrize("S_", [1, 3])
def test_server_short_family(graph14, S_):
    import torch
    t = tpa()
    seeds = synth.query_seeds(graph14["cand"], 7, key=13)
    srv = t.Server(graph14["g"], S_, max_k=8)
    for _ in range(2):
        got = srv.query(seeds).clone()
        assert torch.equal(got, t.query(graph14["g"], seeds, S_))
    parity(got[:, 3].cpu().numpy(), oracle.query(graph14["og"], int(seeds[3]), C, S_, T, graph14["rs"], EPS), "S")
    srv.free()


def test_server_errors(graph14):
    import ctypes
    t = tpa()
    lib = t.library()
    srv = t.Server(graph14["g"], S, max_k=8)
    with pytest.raises(t.TpaError, match="EINVAL"):
        srv.query(np.arange(9, dtype=np.int32))
    with pytest.raises(t.TpaError, match="EINVAL"):
        srv.query([graph14["n"]])
    srv.free()
    g2 = t.build_graph(4, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    h = ctypes.c_void_p()
    st = lib.tpa_server_create(g2.handle, S, 4, None, 0, None, ctypes.byref(h))
    assert t.tpa.STATUS[st] == "TPA_ESTATE"
    host_out = np.zeros((graph14["n"], 4), np.float32)
    st = lib.tpa_server_create(graph14["g"].handle, S, 4, ctypes.c_void_p(host_out.ctypes.data), 4, None,
                               ctypes.byref(h))
    assert t.tpa.STATUS[st] == "TPA_EINVAL"


def test_server_heavy_seeds_and_branch_keys(graph14):
    """Batches whose heavy seeds (more than 256 out-edges) sit at different
    places: the server regroups them like tpa_query (bit-equal results), and
    two batches with the same chunk branches share one captured graph."""
    import torch
    t = tpa()
    og = graph14["og"]
    heavy = np.flatnonzero(og.outdeg > 256).astype(np.int32)
    light = graph14["cand"][og.outdeg[graph14["cand"]] <= 256]
    assert len(heavy) >= 2, "the scale-14 graph has nodes of more than 256 out-edges"
    srv = t.Server(graph14["g"], S, max_k=64)
    a = light[:32].copy()
    a[3] = heavy[0]                 # one heavy seed in the first chunk
    b = light[32:64].copy()
    b[10] = heavy[1]                # one heavy seed in the second chunk: same branches after regrouping
    for sd in (a, b, a):
        got = srv.query(sd).clone()
        assert torch.equal(got, t.query(graph14["g"], sd, S))
    st = srv.stats(32)
    assert st["captures"] == 1 and st["replays"] == 2, st
    parity(got[:, 3].cpu().numpy(), oracle.query(og, int(a[3]), C, S, T, graph14["rs"], EPS), "heavy seed column")
    srv.sync()
    srv.free()
