"""Host logic of query chunking: the order tpa_query runs a query's seeds in
(tpa_seed_order; no GPU needed).

Seeds with more out-edges than the push branch takes (256) make their whole
chunk pull x1 and x2, so tpa_query swaps them into the last places of the
query.  Checked on seeded random degree mixes: the order is a permutation made
of disjoint swaps, every heavy seed ends in the last places, light seeds move
only to fill the places the heavy ones left, and nothing moves when no chunk
can push (push off, S < 4, chunks wider than 16) or the query is one chunk.
"""
import numpy as np
import pytest

import synth


def tpa():
    m = pytest.importorskip("paper_1708_02574_gb300")
    try:
        m.library()
    except Exception as e:   # the library has not been built here
        pytest.skip(f"libtpa not available: {e}")
    return m


def degrees(k, frac_heavy, key):
    u = np.array([synth.uniform(key, i) for i in range(2 * k)])
    od = np.where(u[:k] < frac_heavy, 257 + (u[k:] * 5000).astype(np.int64), (u[k:] * 256).astype(np.int64))
    return od.astype(np.int32)


@pytest.mark.parametrize("k,frac,key", [(1000, 0.017, 41), (40, 0.1, 42), (257, 0.3, 43), (9, 0.5, 44)])
def test_order_moves_heavy_seeds_last(k, frac, key):
    t = tpa()
    od = degrees(k, frac, key)
    perm = t.seed_order(od, S=5)
    assert sorted(perm.tolist()) == list(range(k))
    heavy = od > 256
    nh = int(heavy.sum())
    assert heavy[perm[k - nh:]].all() and not heavy[perm[:k - nh]].any()
    moved = np.flatnonzero(perm != np.arange(k))
    # disjoint swaps: each moved place holds the seed of the place that holds its own
    assert all(perm[perm[j]] == j for j in moved)
    # a light seed moves only out of the last nh places, a heavy one only into them
    for j in moved:
        assert (j >= k - nh) == heavy[perm[j]]


def test_order_is_identity_when_nothing_can_push():
    t = tpa()
    od = degrees(64, 0.2, 45)
    ident = np.arange(64)
    assert not np.array_equal(t.seed_order(od, S=5), ident)
    assert np.array_equal(t.seed_order(od, S=3), ident)          # family of 2 products: no push branch
    assert np.array_equal(t.seed_order(od[:8], S=5), np.arange(8))   # one chunk
    assert np.array_equal(t.seed_order(np.full(20, 300, np.int32), S=5), np.arange(20))   # all heavy
    try:
        t.set_push(False)
        assert np.array_equal(t.seed_order(od, S=5), ident)
        t.set_push(True)
        t.set_batch_width(32)                                     # chunks wider than the push branch takes
        assert np.array_equal(t.seed_order(od, S=5), ident)
    finally:
        t.set_push(True)
        t.set_batch_width(0)


def test_order_rejects_bad_input():
    t = tpa()
    with pytest.raises(t.TpaError, match="EINVAL"):
        t.seed_order(np.zeros(0, np.int32))
