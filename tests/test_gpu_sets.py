"""Seed-set queries (tpa_query_sets) against the FP64 oracle.

Personalised PageRank with the seed vector q_s = 1/|S| of Section II-C through
the batched path: R-MAT scale 14 (16,384 nodes, edge factor 16, key 1), 12 sets
(two query chunks of the default width 8, the second ragged) of 1 to 300
members drawn uniformly over nodes with an out-edge (key 30), with the biggest
hub, a node without out-edges and a repeated member among them.  Every column
within L1 <= 1e-5 and max-abs <= 1e-7 of oracle.query_set, in both product
modes; a one-member set agrees with tpa_query on that seed to the same bars,
and a set with the mean of its members' single-seed columns.
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
    assert np.isfinite(diff).all(), tag
    assert diff.sum() <= 1e-5 and diff.max() <= 1e-7, f"{tag}: L1 {diff.sum():.3e} max {diff.max():.3e}"


@pytest.fixture(scope="module")
def rmat14():
    n = 1 << 14
    s, d = synth.rmat_edges(14, 16)
    og = oracle.build_graph(n, s, d)
    g = tpa().build_graph(n, s, d)
    tpa().preprocess(g, C, T, EPS)
    rs, _ = oracle.preprocess(og, C, T, EPS)
    cand = synth.nodes_with_out_edge(n, s, d)
    dead = np.setdiff1d(np.arange(n), cand)
    return dict(n=n, og=og, g=g, rs=rs, cand=cand, dead=dead)


def make_sets(rmat14):
    pool = synth.query_seeds(rmat14["cand"], 2000, key=30)
    sizes = [1, 3, 2, 17, 300, 5, 1, 8, 40, 2, 9, 4]
    sets, off = [], 0
    for k in sizes:
        sets.append([int(v) for v in pool[off:off + k]])
        off += k
    sets[1][0] = 0                               # the biggest hub
    sets[3][2] = int(rmat14["dead"][0])          # a node without out-edges
    sets[5][4] = sets[5][1]                      # a repeated member counts twice
    return sets


@pytest.mark.parametrize("pattern", [True, False], ids=["pattern", "valued"])
def test_query_sets_parity(rmat14, pattern):
    t = tpa()
    sets = make_sets(rmat14)
    try:
        t.set_pattern(pattern)
        out = t.query_sets(rmat14["g"], sets, S).cpu().numpy()
    finally:
        t.set_pattern(True)
    assert out.shape == (rmat14["n"], len(sets))
    for j, members in enumerate(sets):
        ref = oracle.query_set(rmat14["og"], members, C, S, T, rmat14["rs"], EPS)
        parity(out[:, j], ref, f"pattern={pattern} set {j} ({len(members)} members)")


def test_query_sets_linearity(rmat14):
    t = tpa()
    sets = make_sets(rmat14)
    out = t.query_sets(rmat14["g"], sets, S).cpu().numpy().astype(np.float64)
    one = t.query(rmat14["g"], np.array([sets[0][0]], np.int32), S).cpu().numpy()[:, 0]
    parity(out[:, 0], one.astype(np.float64), "one-member set vs tpa_query")
    members = sets[7]
    singles = t.query(rmat14["g"], np.array(members, np.int32), S).cpu().numpy().astype(np.float64)
    parity(out[:, 7], singles.mean(axis=1), "set vs mean of its members' columns")


def test_query_sets_errors(rmat14):
    import ctypes
    t = tpa()
    with pytest.raises(t.TpaError, match="EINVAL"):
        t.query_sets(rmat14["g"], [[0], []], S)                  # an empty set
    with pytest.raises(t.TpaError, match="EINVAL"):
        t.query_sets(rmat14["g"], [[0, rmat14["n"]]], S)         # a member out of range
    g2 = t.build_graph(4, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    with pytest.raises(t.TpaError, match="ESTATE"):
        t.query_sets(g2, [[0]], S)
    lib = t.library()
    ptr = np.array([0, 1], np.int64)
    mem = np.array([0], np.int32)
    host_out = np.zeros(rmat14["n"], np.float32)
    st = lib.tpa_query_sets(rmat14["g"].handle, ctypes.c_void_p(ptr.ctypes.data), ctypes.c_void_p(mem.ctypes.data),
                            1, S, ctypes.c_void_p(host_out.ctypes.data), None)
    assert t.tpa.STATUS[st] == "TPA_EINVAL"
