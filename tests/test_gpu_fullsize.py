"""Parity at the benchmark's full size, in the launch configuration bench.py times.

R-MAT scale 22 (4,194,304 nodes, 67,108,864 raw edges, key 1), c = 0.15, S = 5,
T = 10, eps = 1e-9: the whole r~_stranger vector of preprocessing, and sampled
columns of one 1,000-seed query batch (seeds uniform over nodes with an out-edge,
key 2; default chunk width, kernel variants and push path) against the FP64
oracle, each within L1 <= 1e-5 and max-abs <= 1e-7.  The oracle needs about a
minute of one host core for the graph and preprocessing, then ~1 s per column.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

C, S, T, EPS = 0.15, 5, 10, 1e-9
SCALE, QUERIES = 22, 1000


def parity(gpu, ref, tag):
    diff = np.abs(np.asarray(gpu, np.float64) - ref)
    assert np.isfinite(diff).all(), tag
    assert diff.sum() <= 1e-5 and diff.max() <= 1e-7, f"{tag}: L1 {diff.sum():.3e} max {diff.max():.3e}"
    return float(diff.sum()), float(diff.max())


@pytest.fixture(scope="module")
def full():
    import torch
    import paper_1708_02574_gb300 as tpa
    n = 1 << SCALE
    s, d = synth.rmat_edges(SCALE, 16)
    g = tpa.build_graph(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    tpa.preprocess(g, C, T, EPS)
    og = oracle.build_graph(n, s, d)
    rs, it = oracle.preprocess(og, C, T, EPS)
    cand = synth.nodes_with_out_edge(n, s, d)
    seeds = synth.query_seeds(cand, QUERIES)
    return dict(n=n, g=g, og=og, rs=rs, it=it, seeds=seeds, tpa=tpa, torch=torch)


def test_fullsize_csr_counts(full):
    assert full["g"].m == full["og"].m
    rp, _, _ = full["tpa"].get_csr(full["g"], 0)
    assert np.array_equal(rp.cpu().numpy(), full["og"].rp_t)


def test_fullsize_preprocess(full):
    r, it = full["tpa"].get_stranger(full["g"])
    parity(r.cpu().numpy(), full["rs"], "r_stranger scale 22")
    assert abs(it - full["it"]) <= 1


def test_fullsize_query_batch(full):
    tpa, torch = full["tpa"], full["torch"]
    seeds = full["seeds"]
    out = tpa.query(full["g"], torch.from_numpy(seeds).cuda(), S)
    cols = [0, 1, 7, 8, 333, 500, 998, 999]      # chunk edges and interiors of the default width
    for j in cols:
        ref = oracle.query(full["og"], int(seeds[j]), C, S, T, full["rs"], EPS)
        parity(out[:, j].cpu().numpy(), ref, f"scale 22 batch column {j} seed {seeds[j]}")


def test_fullsize_server_growing_batches(full):
    """Batched serving on the full-size graph with batch sizes whose workspace
    grows (width-1 chunks, then chunks of 8): every batch equals tpa_query (bit
    for bit unless tpa_query regroups heavy seeds), and graphs captured over
    reallocated buffers are never replayed."""
    tpa, torch = full["tpa"], full["torch"]
    seeds = full["seeds"]
    sizes = [1, 256, 1, 7, 256, 100, 1, 7]
    srv = tpa.Server(full["g"], S, max_k=256)
    off = 0
    for k in sizes:
        sd = seeds[off:off + k]
        off += k
        got = srv.query(torch.from_numpy(sd).cuda()).clone()
        srv.sync()
        ref = tpa.query(full["g"], sd, S)
        tpa.sync(full["g"])
        d = (got.double() - ref.double()).abs()
        assert torch.equal(got, ref), (k, float(d.max()), int((d > 0).sum()))
    st = srv.stats()
    assert st["replays"] + st["captures"] == len(sizes) and st["replays"] >= 2
    j = 3
    ref = oracle.query(full["og"], int(seeds[off - sizes[-1] + j]), C, S, T, full["rs"], EPS)
    parity(got[:, j].cpu().numpy(), ref, "server scale 22")
    srv.free()


# ---------------------------------------------------------------------------
# The batched-serving graph at full size: R-MAT scale 24 (16,777,216 nodes,
# 268,435,456 raw edges, key 1): the whole r~_stranger vector of
# preprocessing against the oracle, and the 8,192-seed stream of uneven
# request batches (sizes uniform over {1, 7, 32, 100, 256}, key 3; seeds
# uniform over nodes with an out-edge, key 2) answered by tpa_query.

SCALE24, SEEDS24 = 24, 8192


@pytest.fixture(scope="module")
def full24():
    import torch
    import paper_1708_02574_gb300 as tpa
    n = 1 << SCALE24
    s, d = synth.rmat_edges(SCALE24, 16)
    g = tpa.build_graph(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    tpa.preprocess(g, C, T, EPS)
    og = oracle.build_graph(n, s, d)
    cand = synth.nodes_with_out_edge(n, s, d)
    del s, d
    rs, it = oracle.preprocess(og, C, T, EPS)
    seeds = synth.query_seeds(cand, SEEDS24)
    sizes = synth.batch_sizes(SEEDS24)
    return dict(n=n, g=g, og=og, rs=rs, it=it, seeds=seeds, sizes=sizes, tpa=tpa, torch=torch)


def test_scale24_preprocess(full24):
    r, it = full24["tpa"].get_stranger(full24["g"])
    parity(r.cpu().numpy(), full24["rs"], "r_stranger scale 24")
    assert abs(it - full24["it"]) <= 1


def test_scale24_uneven_batches(full24):
    """Every batch of the stream: the bounds of Lemma 2 and Theorem 2 on each
    column (the seed's own score is at least (1+alpha)c, scores are
    non-negative, sum to at most 1 and are at least r~_stranger); the first
    and last column of one batch of each size against the FP64 oracle."""
    tpa, torch = full24["tpa"], full24["torch"]
    g, seeds, sizes = full24["g"], full24["seeds"], full24["sizes"]
    assert sum(sizes) == SEEDS24 and set(sizes[:-1]) == {1, 7, 32, 100, 256}   # the last one is truncated
    r_str, _ = tpa.get_stranger(g)
    alpha = ((1 - C) ** S - (1 - C) ** T) / (1 - (1 - C) ** S)
    off, checked = 0, set()
    for b, k in enumerate(sizes):
        sd = seeds[off:off + k]
        off += k
        out = tpa.query(g, torch.from_numpy(sd).cuda(), S)
        assert out.shape == (full24["n"], k)
        own = out[torch.from_numpy(sd).long().cuda(), torch.arange(k, device="cuda")]
        assert bool((own >= (1 + alpha) * C - 1e-6).all()), b
        for j0 in range(0, k, 32):
            blk = out[:, j0:j0 + 32]
            assert bool((blk >= r_str[:, None] - 1e-7).all()), b
            assert bool((blk.double().sum(0) <= 1.0 + 1e-5).all()), b
        if k not in checked:
            checked.add(k)
            for j in sorted({0, k - 1}):
                ref = oracle.query(full24["og"], int(sd[j]), C, S, T, full24["rs"], EPS)
                parity(out[:, j].cpu().numpy(), ref, f"scale 24 batch {b} (k={k}) column {j}")
        del out
    assert off == SEEDS24 and checked == set(sizes)


def test_scale24_server_stream(full24):
    """The batched-serving workload as such: the 8,192-seed stream of uneven
    batches answered by tpa_server replaying CUDA graphs on the scale-24
    graph.  Each batch's own-seed scores meet Lemma 2's bound; one batch of
    each size equals tpa_query bit for bit and its first and last columns are
    within the oracle tolerance; no bounded device wait gave up."""
    tpa, torch = full24["tpa"], full24["torch"]
    g, seeds, sizes = full24["g"], full24["seeds"], full24["sizes"]
    alpha = ((1 - C) ** S - (1 - C) ** T) / (1 - (1 - C) ** S)
    srv = tpa.Server(g, S, max_k=256)
    off, checked = 0, set()
    for b, k in enumerate(sizes):
        sd = seeds[off:off + k]
        off += k
        got = srv.query(torch.from_numpy(sd).cuda())
        own = got[torch.from_numpy(sd).long().cuda(), torch.arange(k, device="cuda")]
        assert bool((own >= (1 + alpha) * C - 1e-6).all()), b
        if k not in checked:
            checked.add(k)
            got = got.clone()
            srv.sync()
            ref = tpa.query(g, sd, S)
            assert torch.equal(got, ref), (b, k)
            for j in sorted({0, k - 1}):
                r = oracle.query(full24["og"], int(sd[j]), C, S, T, full24["rs"], EPS)
                parity(got[:, j].cpu().numpy(), r, f"server scale 24 batch {b} (k={k}) column {j}")
            del ref
    srv.sync()
    st = srv.stats()
    assert st["replays"] + st["captures"] == len(sizes) and st["replays"] > st["captures"], st
    assert checked == set(sizes)
    srv.free()


# ---------------------------------------------------------------------------
# Billion-edge graph: R-MAT scale 26, edge factor 28 (67,108,864 nodes,
# 1,879,048,192 raw edges, key 1), preprocessing and one batch of 64 queries
# (seeds uniform over nodes with an out-edge, key 2).  Properties that hold at
# any size (CSR invariants and sampled rows against the raw edge list, bounds
# of Lemma 2 / Theorem 2, push against pull branch, batched against
# single-seed), and the FP64 oracle on the host's cores (CSR(A~^T) only,
# about 25 GB of host memory): the whole r~_stranger vector and sampled query
# columns element-wise at L1 <= 1e-5 and max-abs <= 1e-7.

SCALE26, EF26, SEEDS26 = 26, 28, 64


@pytest.fixture(scope="module")
def big26():
    import torch
    import paper_1708_02574_gb300 as tpa
    n = 1 << SCALE26
    torch.cuda.empty_cache()
    s, d = synth.rmat_edges(SCALE26, EF26)
    g = tpa.build_graph(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    torch.cuda.empty_cache()
    tpa.preprocess(g, C, T, EPS)
    cand = synth.nodes_with_out_edge(n, s, d)
    seeds = synth.query_seeds(cand, SEEDS26)
    return dict(n=n, s=s, d=d, g=g, seeds=seeds, tpa=tpa, torch=torch)


def test_scale26_csr_invariants(big26):
    tpa, torch = big26["tpa"], big26["torch"]
    g, n = big26["g"], big26["n"]
    rp_t, col_t, val_t = tpa.get_csr(g, 0)
    rp_a, _, _ = tpa.get_csr(g, 1)
    m = g.m
    assert m > 10 ** 9 and int(rp_t[-1]) == m and int(rp_a[-1]) == m
    assert bool((rp_t[1:] >= rp_t[:-1]).all()) and bool((rp_a[1:] >= rp_a[:-1]).all())
    assert int(col_t.min()) >= 0 and int(col_t.max()) < n
    outdeg = (rp_a[1:] - rp_a[:-1]).to(torch.float64)
    # val = RN32(1 / outdeg(source)) on every edge of CSR(A~^T), in slices
    step = 1 << 27
    for e0 in range(0, m, step):
        c = col_t[e0:e0 + step].long()
        assert torch.equal(val_t[e0:e0 + step], (1.0 / outdeg[c]).to(torch.float32)), e0
    del c
    # sampled destination rows: strictly increasing sources, no self-loop, and
    # exactly the distinct sources of the raw edges into that row
    rng = np.random.default_rng(26)
    rows = [0, 1] + [int(r) for r in rng.integers(0, n, 2)]
    s, d = big26["s"], big26["d"]
    rp = rp_t.cpu().numpy()
    for v in rows:
        got = col_t[int(rp[v]):int(rp[v + 1])].cpu().numpy()
        assert np.all(np.diff(got) > 0) and not np.any(got == v)
        raw = s[d == v]
        assert np.array_equal(got, np.unique(raw[raw != v])), v


def test_scale26_preprocess_bounds(big26):
    tpa = big26["tpa"]
    r, it = tpa.get_stranger(big26["g"])
    assert bool((r >= 0).all())
    mass = float(r.double().sum())
    assert 0.0 < mass <= (1 - C) ** T + 1e-6       # Lemma 2 with mass lost at deadends
    assert 0 < it <= 130


def test_scale26_batched_queries(big26):
    tpa, torch = big26["tpa"], big26["torch"]
    g, seeds = big26["g"], big26["seeds"]
    r_str, _ = tpa.get_stranger(g)
    out = tpa.query(g, seeds, S)
    alpha = ((1 - C) ** S - (1 - C) ** T) / (1 - (1 - C) ** S)
    own = out[torch.from_numpy(seeds).long().cuda(), torch.arange(len(seeds), device="cuda")]
    assert bool((own >= (1 + alpha) * C - 1e-6).all())               # x0 = c e_s alone
    for j0 in range(0, len(seeds), 8):                                # column blocks bound the memory
        blk = out[:, j0:j0 + 8]
        assert bool((blk >= 0).all())
        assert bool((blk.double().sum(0) <= 1.0 + 1e-5).all())
        assert bool((blk >= r_str[:, None] - 1e-7).all())            # the family part is non-negative
    try:
        tpa.set_push(False)
        pulled = tpa.query(g, seeds, S)
    finally:
        tpa.set_push(True)
    for j0 in range(0, len(seeds), 8):
        diff = (out[:, j0:j0 + 8].double() - pulled[:, j0:j0 + 8].double()).abs()
        assert float(diff.sum(0).max()) <= 1e-5 and float(diff.max()) <= 1e-7, j0
    del pulled, diff
    one = tpa.query(g, seeds[5:6], S)
    d1 = (one[:, 0].double() - out[:, 5].double()).abs()
    assert float(d1.sum()) <= 1e-5 and float(d1.max()) <= 1e-7


@pytest.fixture(scope="module")
def oracle26(big26):
    og = oracle.build_graph(big26["n"], big26["s"], big26["d"], with_a=False)
    rs, it = oracle.preprocess(og, C, T, EPS)
    return dict(og=og, rs=rs, it=it)


def test_scale26_preprocess_oracle(big26, oracle26):
    """Algorithm 2 on the billion-edge graph: GPU FP32 against the FP64 oracle."""
    tpa = big26["tpa"]
    assert big26["g"].m == oracle26["og"].m
    r, it = tpa.get_stranger(big26["g"])
    parity(r.cpu().numpy(), oracle26["rs"], "r_stranger scale 26")
    assert abs(it - oracle26["it"]) <= 1


def test_scale26_query_columns_oracle(big26, oracle26):
    """Algorithm 3 on the billion-edge graph: the first and last columns of the
    64-seed batch against the FP64 oracle."""
    tpa = big26["tpa"]
    seeds = big26["seeds"]
    out = tpa.query(big26["g"], seeds, S)
    for j in (0, len(seeds) - 1):
        ref = oracle.query(oracle26["og"], int(seeds[j]), C, S, T, oracle26["rs"], EPS)
        parity(out[:, j].cpu().numpy(), ref, f"scale 26 column {j} seed {seeds[j]}")
