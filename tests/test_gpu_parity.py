"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars: CSR bit-exact; every FP32 score vector within
L1 <= 1e-5 and max-abs <= 1e-7 of the FP64 oracle, checked per result.
Graphs: R-MAT scale 14 (16,384 nodes, edge factor 16, a/b/c/d = .57/.19/.19/.05,
key 1) plus small named graphs; the merge-path tiles there span many tiles and
end in a ragged tail.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

C, S, T, EPS = 0.15, 5, 10, 1e-9
L1_TOL, MAX_TOL = 1e-5, 1e-7


def tpa():
    import paper_1708_02574_gb300 as m
    return m


def parity(gpu, ref, tag=""):
    g = np.asarray(gpu, dtype=np.float64)
    diff = np.abs(g - ref)
    l1, mx = float(diff.sum()), float(diff.max()) if diff.size else 0.0
    assert np.isfinite(g).all(), tag
    assert l1 <= L1_TOL and mx <= MAX_TOL, f"{tag}: L1 {l1:.3e} max-abs {mx:.3e}"
    return l1, mx


@pytest.fixture(scope="module")
def rmat14():
    s, d = synth.rmat_edges(14, 16)
    n = 1 << 14
    og = oracle.build_graph(n, s, d)
    g = tpa().build_graph(n, s, d)
    rs, it = oracle.preprocess(og, C, T, EPS)
    tpa().preprocess(g, C, T, EPS)
    cand = synth.nodes_with_out_edge(n, s, d)
    return dict(n=n, s=s, d=d, og=og, g=g, rs=rs, it=it, cand=cand)


def csr_equal(g, og):
    t = tpa()
    for which, (rp, col, val) in ((0, (og.rp_t, og.col_t, og.val_t)), (1, (og.rp_a, og.col_a, og.val_a))):
        grp, gcol, gval = (a.cpu().numpy() for a in t.get_csr(g, which))
        assert np.array_equal(grp, rp), which
        assert np.array_equal(gcol, col), which
        # RN32(1/outdeg) equals the FP32 rounding of the exact FP64 1/outdeg for outdeg < 2^24
        assert np.array_equal(gval.view(np.uint32), val.astype(np.float32).view(np.uint32)), which


def test_csr_bit_exact_rmat14(rmat14):
    assert rmat14["g"].m == rmat14["og"].m
    csr_equal(rmat14["g"], rmat14["og"])


@pytest.mark.parametrize("kind,n", [("cycle", 7), ("star", 33), ("random", 300), ("complete", 12),
                                    ("random_nodead", 1000)])
def test_csr_bit_exact_small(kind, n):
    n, s, d = synth.small_graph(kind, n)
    og = oracle.build_graph(n, s, d)
    g = tpa().build_graph(n, s, d)
    assert g.m == og.m
    csr_equal(g, og)


def test_csr_degenerate():
    t = tpa()
    g = t.build_graph(1, np.zeros(3, np.int32), np.zeros(3, np.int32))   # only self-loops
    assert (g.n, g.m) == (1, 0)
    g = t.build_graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32))   # no edges
    assert (g.n, g.m) == (5, 0)
    rp, _, _ = t.get_csr(g, 0)
    assert rp.cpu().tolist() == [0] * 6
    t.preprocess(g, C, T, EPS)
    out = t.query(g, [2, 4], S).cpu().numpy()
    og = oracle.build_graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    rs, _ = oracle.preprocess(og, C, T, EPS)
    for j, sd in enumerate([2, 4]):
        parity(out[:, j], oracle.query(og, sd, C, S, T, rs, EPS), f"empty graph seed {sd}")


def test_preprocess_parity(rmat14):
    r, it = tpa().get_stranger(rmat14["g"])
    parity(r.cpu().numpy(), rmat14["rs"], "r_stranger")
    assert abs(it - rmat14["it"]) <= 1, (it, rmat14["it"])


@pytest.mark.parametrize("k", [1, 7, 32, 100, 256, 300])
def test_query_parity(rmat14, k):
    cand = rmat14["cand"]
    seeds = synth.query_seeds(cand, k, key=2)
    seeds[0] = 0                                   # the biggest hub
    if k > 2:
        dead = np.setdiff1d(np.arange(rmat14["n"]), cand)
        seeds[1] = dead[0]                         # a node without out-edges
    out = tpa().query(rmat14["g"], seeds, S).cpu().numpy()
    assert out.shape == (rmat14["n"], k)
    cols = range(k) if k <= 32 else list(range(8)) + list(range(k - 8, k))
    for j in cols:
        ref = oracle.query(rmat14["og"], int(seeds[j]), C, S, T, rmat14["rs"], EPS)
        parity(out[:, j], ref, f"k={k} col {j} seed {seeds[j]}")


def test_query_matches_single_seed_columns(rmat14):
    """A batched query agrees with single-seed queries column by column (parity tolerance)."""
    t = tpa()
    seeds = synth.query_seeds(rmat14["cand"], 7, key=9)
    batch = t.query(rmat14["g"], seeds, S).cpu().numpy()
    for j in (0, 3, 6):
        one = t.query(rmat14["g"], seeds[j:j + 1], S).cpu().numpy()[:, 0]
        parity(batch[:, j], one.astype(np.float64), f"column {j}")


@pytest.mark.parametrize("S_", [1, 2, 10])
def test_query_edge_S(rmat14, S_):
    seeds = np.array([0, 5, int(rmat14["cand"][-1])], np.int32)
    out = tpa().query(rmat14["g"], seeds, S_).cpu().numpy()
    for j, sd in enumerate(seeds):
        parity(out[:, j], oracle.query(rmat14["og"], int(sd), C, S_, T, rmat14["rs"], EPS), f"S={S_} seed {sd}")


def test_cpi_exact_parity(rmat14):
    for sd in (0, int(rmat14["cand"][len(rmat14["cand"]) // 2])):
        out, it = tpa().cpi_exact(rmat14["g"], sd, C, EPS)
        ref, rit = oracle.cpi_exact(rmat14["og"], sd, C, EPS)
        parity(out.cpu().numpy(), ref, f"exact CPI seed {sd}")
        assert abs(it - rit) <= 1


def test_cpi_parts_parity(rmat14):
    """Algorithm 1 with s_iter/t_iter: neighbor part (S..T-1) and stranger part (T..inf)."""
    seeds = np.array([0, 17, int(rmat14["cand"][3])], np.int32)
    for s_it, t_it in ((S, T - 1), (T, -1), (0, 0), (3, 3)):
        out, iters = tpa().cpi(rmat14["g"], seeds, C, EPS, s_it, t_it)
        out = out.cpu().numpy()
        for j, sd in enumerate(seeds):
            q = np.zeros(rmat14["n"])
            q[sd] = 1.0
            ref, rit = oracle.cpi(rmat14["og"], q, C, EPS, s_it, None if t_it < 0 else t_it)
            parity(out[:, j], ref, f"cpi({s_it},{t_it}) seed {sd}")
            assert abs(int(iters[j]) - rit) <= 1


def test_host_buffers_through_c_abi(rmat14):
    """Host input and output pointers: the library copies in and out itself."""
    import ctypes
    t = tpa()
    lib = t.library()
    seeds = np.array([0, 11, 99], np.int32)
    out = np.empty((rmat14["n"], 3), np.float32)
    st = lib.tpa_query(rmat14["g"].handle, ctypes.c_void_p(seeds.ctypes.data), 3, S,
                       ctypes.c_void_p(out.ctypes.data), None)
    assert st == 0, lib.tpa_last_error()
    dev = t.query(rmat14["g"], seeds, S).cpu().numpy()
    assert np.array_equal(out, dev)


@pytest.mark.parametrize("k,group", [(13, -1), (152, -1), (150, 72), (600, 256), (600, 0)])
def test_pinned_host_output(rmat14, k, group):
    """Page-locked host output: the kernels write the scores straight into it
    (152 columns: 16-byte rows), or it is staged in device memory and copied
    once (13 columns: rows not 16-byte aligned), or column groups are computed
    in device buffers and copied while the next group computes (150 columns
    in groups of 72: three groups, the third reusing the first one's buffer;
    600 in groups of 256; 600 with the default groups of 128)."""
    import torch
    t = tpa()
    seeds = synth.query_seeds(rmat14["cand"], k, key=14)
    out = torch.full((rmat14["n"], k), -1.0, dtype=torch.float32).pin_memory()
    t.set_output_group_width(group)
    try:
        t.query(rmat14["g"], seeds, S, out=out)
    finally:
        t.set_output_group_width(0)
    dev = t.query(rmat14["g"], seeds, S).cpu()
    if k <= 8 or not (rmat14["og"].outdeg[seeds] > 256).any():
        assert torch.equal(out, dev)
    else:   # into device memory tpa_query regroups seeds too heavy to push: FP32 rounding
        d = (out.double() - dev.double()).abs()
        assert float(d.sum(0).max()) <= 1e-5 and float(d.max()) <= 1e-7
    for j in (0, k // 2, k - 1):
        parity(out[:, j].numpy(), oracle.query(rmat14["og"], int(seeds[j]), C, S, T, rmat14["rs"], EPS), f"col {j}")


def test_deterministic(rmat14):
    seeds = synth.query_seeds(rmat14["cand"], 32, key=4)
    a = tpa().query(rmat14["g"], seeds, S).cpu().numpy()
    b = tpa().query(rmat14["g"], seeds, S).cpu().numpy()
    assert np.array_equal(a, b)


def test_errors(rmat14):
    t = tpa()
    with pytest.raises(t.TpaError, match="EINVAL"):
        t.query(rmat14["g"], [rmat14["n"]], S)
    with pytest.raises(t.TpaError, match="EINVAL"):
        t.query(rmat14["g"], [-1], S)
    with pytest.raises(t.TpaError, match="EINVAL"):
        t.query(rmat14["g"], [0], T + 1)
    with pytest.raises(t.TpaError, match="EINVAL"):
        t.preprocess(rmat14["g"], 1.5, T, EPS)
    with pytest.raises(t.TpaError, match="EINVAL"):
        t.build_graph(4, np.array([0, 4], np.int32), np.array([1, 2], np.int32))
    g2 = t.build_graph(4, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    with pytest.raises(t.TpaError, match="ESTATE"):
        t.query(g2, [0], S)


def test_save_load_preprocessed(rmat14, tmp_path):
    t = tpa()
    p = str(tmp_path / "str.bin")
    t.save_preprocessed(rmat14["g"], p)
    g2 = t.build_graph(rmat14["n"], rmat14["s"], rmat14["d"])
    t.load_preprocessed(g2, p)
    a, ia = t.get_stranger(rmat14["g"])
    b, ib = t.get_stranger(g2)
    assert ia == ib and np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    seeds = [0, 3]
    assert np.array_equal(t.query(g2, seeds, S).cpu().numpy(), t.query(rmat14["g"], seeds, S).cpu().numpy())
    small = t.build_graph(5, np.array([0, 1], np.int32), np.array([1, 2], np.int32))
    with pytest.raises(t.TpaError, match="EINVAL"):
        t.load_preprocessed(small, p)


@pytest.fixture
def narrow_batches():
    t = tpa()
    t.set_batch_width(8)
    yield
    t.set_batch_width(0)
    t.set_push(True)


@pytest.mark.parametrize("k,S_", [(1, 5), (3, 4), (8, 5), (8, 10), (13, 6)])
def test_query_push_path(rmat14, narrow_batches, k, S_):
    """Light seeds in chunks of <= 8: x1 and x2 are pushed along CSR(A~); parity with the oracle."""
    n = rmat14["n"]
    og = rmat14["og"]
    light = rmat14["cand"][(og.outdeg[rmat14["cand"]] <= 256)]
    seeds = synth.query_seeds(light, k, key=20 + k)
    if k >= 3:
        dead = np.setdiff1d(np.arange(n), rmat14["cand"])
        seeds[1] = dead[3]                         # no out-edges: the column stops after x1
    out = tpa().query(rmat14["g"], seeds, S_).cpu().numpy()
    for j in range(k):
        ref = oracle.query(og, int(seeds[j]), C, S_, T, rmat14["rs"], EPS)
        parity(out[:, j], ref, f"push k={k} S={S_} col {j} seed {seeds[j]}")
    t = tpa()
    t.set_push(False)
    pulled = t.query(rmat14["g"], seeds, S_).cpu().numpy()
    for j in range(k):
        parity(out[:, j], pulled[:, j].astype(np.float64), f"push vs pull col {j}")


def test_query_push_deterministic(rmat14, narrow_batches):
    light = rmat14["cand"][(rmat14["og"].outdeg[rmat14["cand"]] <= 256)]
    seeds = synth.query_seeds(light, 8, key=31)
    a = tpa().query(rmat14["g"], seeds, S).cpu().numpy()
    b = tpa().query(rmat14["g"], seeds, S).cpu().numpy()
    assert np.array_equal(a, b)


def test_pattern_only_products(rmat14):
    """Pattern-only products (the default: the iterate kept scaled by
    RN32(1/outdeg), the value array not read) and products that read the value
    array give the same TPA scores up to FP32 rounding, each within the bars of
    the oracle, for preprocessing and a query batch; on a weighted graph the
    setting changes nothing."""
    import torch
    t = tpa()
    seeds = synth.query_seeds(rmat14["cand"], 40, key=21)
    seeds[0] = 0                                       # the biggest hub: a pulled chunk
    res = {}
    try:
        for mode in (True, False):
            t.set_pattern(mode)
            t.preprocess(rmat14["g"], C, T, EPS)
            r, it = t.get_stranger(rmat14["g"])
            parity(r.cpu().numpy(), rmat14["rs"], f"r_stranger pattern={mode}")
            assert abs(it - rmat14["it"]) <= 1
            out = t.query(rmat14["g"], seeds, S).cpu().numpy()
            for j in (0, 1, 8, 39):
                ref = oracle.query(rmat14["og"], int(seeds[j]), C, S, T, rmat14["rs"], EPS)
                parity(out[:, j], ref, f"pattern={mode} col {j}")
            res[mode] = out
        d = np.abs(res[True].astype(np.float64) - res[False])
        assert d.sum(0).max() <= 1e-5 and d.max() <= 1e-7

        n = 1 << 10
        s, dst = synth.rmat_edges(10, 16)
        g = t.build_graph(n, s, dst)
        w = torch.from_numpy(synth.normal(g.m, key=4)).cuda().exp()
        t.set_edge_weights(g, w)
        sd = synth.query_seeds(synth.nodes_with_out_edge(n, s, dst), 8, key=22)
        outs = []
        for mode in (True, False):
            t.set_pattern(mode)
            t.preprocess(g, C, T, EPS)
            outs.append(t.query(g, sd, S).clone())
        assert torch.equal(outs[0], outs[1])
    finally:
        t.set_pattern(True)
        t.preprocess(rmat14["g"], C, T, EPS)


def test_heavy_seeds_grouped(rmat14):
    """Seeds with more out-edges than the push branch takes are moved to the
    last chunks of a query, so only those chunks pull x1 and x2: 40 seeds with
    three heavy ones spread over three chunks take 12 SpMM launches instead of
    16, and every column lands where its seed was (parity with the oracle)."""
    t = tpa()
    og = rmat14["og"]
    cand = rmat14["cand"]
    light = cand[og.outdeg[cand] <= 256]
    heavy = cand[og.outdeg[cand] > 256]
    assert heavy.size >= 3
    seeds = synth.query_seeds(light, 40, key=23)
    for pos, h in zip((2, 17, 30), heavy[:3]):
        seeds[pos] = h
    t.profile_reset(True)
    out = t.query(rmat14["g"], seeds, S).cpu().numpy()
    spmm = sum(v["launches"] for k2, v in t.profile_read().items() if k2.startswith("spmm"))
    t.profile_reset(False)
    assert spmm == 4 * 1 + 2 * 4, spmm
    for j in (0, 2, 3, 17, 30, 36, 37, 38, 39):
        ref = oracle.query(og, int(seeds[j]), C, S, T, rmat14["rs"], EPS)
        parity(out[:, j], ref, f"grouped col {j} seed {seeds[j]}")
    try:
        t.set_push(False)                       # no push branch: nothing is regrouped
        pulled = t.query(rmat14["g"], seeds, S).cpu().numpy()
    finally:
        t.set_push(True)
    d = np.abs(out.astype(np.float64) - pulled)
    assert d.sum(0).max() <= 1e-5 and d.max() <= 1e-7


def test_results_do_not_depend_on_earlier_calls(rmat14):
    """The iterate buffers of a graph are reused across calls whose padded
    widths differ ([n][8] then [n][1], ...): rows without in-edges, which the
    SpMV/SpMM does not write, must read as zero under every layout.  Each call
    on the long-lived graph equals the same call on a fresh graph bit for bit,
    and the oracle within tolerance."""
    import torch
    t = tpa()
    n, s, d = rmat14["n"], rmat14["s"], rmat14["d"]
    seeds = synth.query_seeds(rmat14["cand"], 64, key=21)
    g = rmat14["g"]
    for k in (8, 1, 4, 2, 8, 3, 1, 16, 1):
        sd = seeds[:k]
        got = t.query(g, sd, S).clone()
        fresh = t.build_graph(n, s, d)
        t.preprocess(fresh, C, T, EPS)
        ref = t.query(fresh, sd, S)
        assert torch.equal(got, ref), k
        parity(got[:, k - 1].cpu().numpy(), oracle.query(rmat14["og"], int(sd[k - 1]), C, S, T, rmat14["rs"], EPS),
               f"k {k}")
        r1, _ = t.cpi(g, sd[:1], C, EPS, 0, 3)
        r2, _ = t.cpi(fresh, sd[:1], C, EPS, 0, 3)
        assert torch.equal(r1, r2), k
        fresh.free()
