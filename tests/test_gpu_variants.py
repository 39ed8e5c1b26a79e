"""Every compiled SpMV/SpMM variant against the FP64 oracle.

The autotuner may pick any variant, so each one is forced in turn and checked
on R-MAT scale 12 (4,096 nodes, edge factor 16, key 1; a few hundred merge-path
tiles with a ragged tail):
  - a TPA query of kp seeds (push path on, light seeds plus the biggest hub and
    a node without out-edges), and the same query pulled only;
  - Algorithm 1 with s_iter/t_iter into a caller buffer of kp - 1 columns (the
    accumulator's row stride differs from the padded width);
  - preprocessing for the width-1 variants;
each with pattern-only products (the default: x kept scaled by 1/outdeg, no
value array read) and with products that read the value array.
Bars as in the other parity tests: L1 <= 1e-5 and max-abs <= 1e-7 per result.
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
def rmat12():
    n = 1 << 12
    s, d = synth.rmat_edges(12, 16)
    og = oracle.build_graph(n, s, d)
    g = tpa().build_graph(n, s, d)
    rs, it = oracle.preprocess(og, C, T, EPS)
    tpa().preprocess(g, C, T, EPS)
    cand = synth.nodes_with_out_edge(n, s, d)
    light = cand[og.outdeg[cand] <= 256]
    dead = np.setdiff1d(np.arange(n), cand)
    return dict(n=n, og=og, g=g, rs=rs, it=it, cand=cand, light=light, dead=dead)


def variant_ids():
    try:
        return [v["index"] for v in tpa().variants()]
    except Exception:       # no library or no GPU: the tests skip at collection time
        return [0]


@pytest.fixture
def forced(request):
    t = tpa()
    v = t.variants()[request.param]
    t.set_variant(v["kp"], v["index"])
    t.set_batch_width(v["kp"])
    t.set_cpi_batch_width(v["kp"])
    yield v
    t.set_variant(v["kp"], -1)
    t.set_batch_width(0)
    t.set_cpi_batch_width(0)
    t.set_push(True)


@pytest.fixture(params=[True, False], ids=["pattern", "valued"])
def pattern(request):
    tpa().set_pattern(request.param)
    yield request.param
    tpa().set_pattern(True)


def columns(k):
    return range(k) if k <= 16 else sorted({0, 1, 2, k // 2, k - 2, k - 1})


@pytest.mark.parametrize("forced", variant_ids(), indirect=True)
def test_variant_query(rmat12, forced, pattern):
    t = tpa()
    kp = forced["kp"]
    seeds = synth.query_seeds(rmat12["light"], kp, key=40 + kp)
    seeds[0] = 0                                  # the biggest hub: this chunk is pulled
    if kp >= 2:
        seeds[-1] = rmat12["dead"][1]              # stops after x0
    for push in (True, False):
        t.set_push(push)
        out = t.query(rmat12["g"], seeds, S).cpu().numpy()
        for j in columns(kp):
            ref = oracle.query(rmat12["og"], int(seeds[j]), C, S, T, rmat12["rs"], EPS)
            parity(out[:, j], ref, f"{forced['name']} push={push} col {j} seed {seeds[j]}")
    if kp <= 8:
        # a chunk of light seeds only takes the push path for x1 and x2
        t.set_push(True)
        light = synth.query_seeds(rmat12["light"], kp, key=60 + kp)
        out = t.query(rmat12["g"], light, S).cpu().numpy()
        again = t.query(rmat12["g"], light, S).cpu().numpy()
        assert np.array_equal(out, again), forced["name"]
        for j in range(kp):
            ref = oracle.query(rmat12["og"], int(light[j]), C, S, T, rmat12["rs"], EPS)
            parity(out[:, j], ref, f"{forced['name']} light col {j}")


@pytest.mark.parametrize("forced", variant_ids(), indirect=True)
def test_variant_cpi_parts(rmat12, forced, pattern):
    t = tpa()
    kp = forced["kp"]
    k = max(1, kp - 1)
    seeds = synth.query_seeds(rmat12["cand"], k, key=80 + kp)
    for s_it, t_it in ((S, T - 1), (0, 3)):
        out, iters = t.cpi(rmat12["g"], seeds, C, EPS, s_it, t_it)
        out = out.cpu().numpy()
        for j in columns(k):
            q = np.zeros(rmat12["n"])
            q[seeds[j]] = 1.0
            ref, _ = oracle.cpi(rmat12["og"], q, C, EPS, s_it, t_it)
            parity(out[:, j], ref, f"{forced['name']} cpi({s_it},{t_it}) col {j}")


@pytest.mark.parametrize("forced", [v for v in variant_ids()], indirect=True)
def test_variant_preprocess(rmat12, forced, pattern):
    if forced["kp"] != 1:
        pytest.skip("preprocessing runs one column")
    t = tpa()
    t.preprocess(rmat12["g"], C, T, EPS)
    r, it = t.get_stranger(rmat12["g"])
    parity(r.cpu().numpy(), rmat12["rs"], f"{forced['name']} r_stranger")
    assert abs(it - rmat12["it"]) <= 1


@pytest.fixture(scope="module")
def rmat17():
    n = 1 << 17
    s, d = synth.rmat_edges(17, 16)
    og = oracle.build_graph(n, s, d)
    g = tpa().build_graph(n, s, d)
    rs, it = oracle.preprocess(og, C, T, EPS)
    return dict(n=n, og=og, g=g, rs=rs, it=it, cand=synth.nodes_with_out_edge(n, s, d))


def segmented_ids():
    """Variants without the merge-path fixup: the segmented walks, the
    pipelined kernel that finishes its deferred rows itself, and the
    lane-segment walk with its finishing launch."""
    try:
        return [v["index"] for v in tpa().variants() if v["name"].startswith(("seg", "pipef", "lane"))]
    except Exception:
        return [0]


@pytest.mark.parametrize("forced", segmented_ids(), indirect=True)
def test_segmented_walk_many_tiles_per_warp(rmat17, forced, pattern):
    """R-MAT scale 17 (about 2 million nonzeros): every warp of the persistent
    grid walks several tiles, so the stage ring, the gathers sent one tile
    ahead, the rows deferred to the warp's next tile and the waits on other
    warps' carry-outs all run."""
    t = tpa()
    kp = forced["kp"]
    if kp == 1:
        t.preprocess(rmat17["g"], C, T, EPS)
        r, it = t.get_stranger(rmat17["g"])
        parity(r.cpu().numpy(), rmat17["rs"], f"{forced['name']} r_stranger")
        assert abs(it - rmat17["it"]) <= 1
        return
    forced_name = forced["name"]
    t.set_variant(kp, -1)
    t.preprocess(rmat17["g"], C, T, EPS)
    t.set_variant(kp, forced["index"])
    seeds = synth.query_seeds(rmat17["cand"], kp, key=90 + kp)
    seeds[0] = 0
    t.set_push(False)
    out = t.query(rmat17["g"], seeds, S).cpu().numpy()
    again = t.query(rmat17["g"], seeds, S).cpu().numpy()
    assert np.array_equal(out, again), forced_name
    if forced_name.startswith("pipef"):
        # the same sums in the same order as the kernel with a fixup launch
        t.set_variant(kp, -1)
        base = t.query(rmat17["g"], seeds, S).cpu().numpy()
        t.set_variant(kp, forced["index"])
        if t.variants()[t.get_variant(kp)]["name"] == forced_name.replace("pipef", "pipe"):
            assert np.array_equal(out, base), forced_name
    for j in sorted({0, kp // 2, kp - 1}):
        ref = oracle.query(rmat17["og"], int(seeds[j]), C, S, T, rmat17["rs"], EPS)
        parity(out[:, j], ref, f"{forced_name} col {j} seed {seeds[j]}")
