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


# ---------------------------------------------------------------------------
# The batched-serving graph at full size: R-MAT scale 24 (16,777,216 nodes,
# 268,435,456 raw edges, key 1): the whole r~_stranger vector of
# preprocessing against the oracle.

SCALE24 = 24


@pytest.fixture(scope="module")
def full24():
    import torch
    import paper_1708_02574_gb300 as tpa
    n = 1 << SCALE24
    s, d = synth.rmat_edges(SCALE24, 16)
    g = tpa.build_graph(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    tpa.preprocess(g, C, T, EPS)
    og = oracle.build_graph(n, s, d)
    del s, d
    rs, it = oracle.preprocess(og, C, T, EPS)
    return dict(n=n, g=g, og=og, rs=rs, it=it, tpa=tpa, torch=torch)


def test_scale24_preprocess(full24):
    r, it = full24["tpa"].get_stranger(full24["g"])
    parity(r.cpu().numpy(), full24["rs"], "r_stranger scale 24")
    assert abs(it - full24["it"]) <= 1
