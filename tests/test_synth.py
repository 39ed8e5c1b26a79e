"""Checks on the seeded input generators (not part of either compute path)."""
import numpy as np

import synth


def _sm64_py(key, ctr):
    M = (1 << 64) - 1
    z = (key + (ctr + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_splitmix64_published_vector():
    # First outputs of the SplitMix64 reference generator seeded with 1234567.
    assert synth.splitmix64(1234567, 0) == 6457827717110365317
    assert synth.splitmix64(1234567, 1) == 3203168211198807973
    for ctr in (0, 5, 1 << 40):
        assert synth.splitmix64(99, ctr) == _sm64_py(99, ctr)


def test_rmat_matches_definition_and_is_thread_independent():
    scale = 10
    s1, d1 = synth.rmat_edges(scale, 4, threads=1)
    s2, d2 = synth.rmat_edges(scale, 4, threads=7)
    assert np.array_equal(s1, s2) and np.array_equal(d1, d2)
    for e in (0, 1, 777, s1.size - 1):
        s = d = 0
        for lvl in range(scale):
            u = (_sm64_py(1, e * scale + lvl) >> 11) * 2.0 ** -53
            sb, db = (0, 0) if u < .57 else (0, 1) if u < .76 else (1, 0) if u < .95 else (1, 1)
            s, d = (s << 1) | sb, (d << 1) | db
        assert (s1[e], d1[e]) == (s, d)


def test_rmat_quadrant_frequencies():
    s, d = synth.rmat_edges(12, 16)
    top_s, top_d = s >> 11, d >> 11
    f = np.bincount(top_s * 2 + top_d, minlength=4) / s.size
    assert np.allclose(f, [.57, .19, .19, .05], atol=0.01)
    assert s.min() >= 0 and s.max() < 4096 and d.max() < 4096


def test_seed_picks_and_sizes():
    s, d = synth.rmat_edges(10, 8)
    n = 1 << 10
    cand = synth.nodes_with_out_edge(n, s, d)
    brute = sorted({int(a) for a, b in zip(s, d) if a != b})
    assert cand.tolist() == brute
    q = synth.query_seeds(cand, 500)
    assert np.isin(q, cand).all()
    sizes = synth.batch_sizes(8192)
    assert sum(sizes) == 8192 and set(sizes[:-1]) <= {1, 7, 32, 100, 256}
    x = synth.normal(20000, 4)
    assert abs(x.mean()) < 0.03 and abs(x.std() - 1) < 0.03
    sd, p, ng = synth.triples(n, s, d, cand, 300)
    edges = set(zip(s.tolist(), d.tolist()))
    assert all((a, b) in edges and a != b for a, b in zip(sd.tolist(), p.tolist()))
    assert ng.min() >= 0 and ng.max() < n


def test_planted_partition_edges():
    """Planted-partition graph: ids in range, the share of edges inside the
    source's block close to p_in plus the uniform draws that land there, and
    the same edges for the same key."""
    n, blocks, p_in = 1 << 12, 64, 0.8
    s, d = synth.planted_edges(n, 16, blocks, p_in)
    assert s.size == d.size == 16 * n
    assert s.min() >= 0 and s.max() < n and d.min() >= 0 and d.max() < n
    inside = (s * blocks // n == d * blocks // n).mean()
    assert abs(inside - (p_in + (1 - p_in) / blocks)) < 0.01
    s2, d2 = synth.planted_edges(n, 16, blocks, p_in)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)
    s3, _ = synth.planted_edges(n, 16, blocks, p_in, key=8)
    assert not np.array_equal(s, s3)
