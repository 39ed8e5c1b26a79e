"""The accuracy study of TPA's approximations (paper_1708_02574_gb300.accuracy).

R-MAT scale 14 (16,384 nodes, edge factor 16, key 1), 6 seeds uniform over
nodes with an out-edge (key 31), (S, T) in {(5, 10), (2, 4), (3, 6), (4, 4)}:
  - each error within its bound (Lemma 3, Lemma 1, Theorem 2; deadends only
    lose mass, so the bounds hold as inequalities);
  - the family, neighbor and stranger parts add up to exact CPI;
  - the three errors match the same quantities computed by the FP64 oracle
    (its CPI parts, preprocessing and Algorithm 3) to 2e-5 absolute: each is
    an L1 norm over 16,384 nodes of FP32 vectors within 1e-5 of the oracle's;
  - recall@100 lies in [0, 1] and within 0.05 of the oracle vectors' recall
    (near-ties at the 100th place may order differently in FP32).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

C, EPS = 0.15, 1e-9
SETTINGS = [(5, 10), (2, 4), (3, 6), (4, 4)]


def tpa():
    import paper_1708_02574_gb300 as m
    return m


@pytest.fixture(scope="module")
def rmat14():
    n = 1 << 14
    s, d = synth.rmat_edges(14, 16)
    og = oracle.build_graph(n, s, d)
    g = tpa().build_graph(n, s, d)
    seeds = synth.query_seeds(synth.nodes_with_out_edge(n, s, d), 6, key=31)
    return dict(n=n, og=og, g=g, seeds=seeds)


def oracle_errors(og, seeds, S, T, k=100):
    n = og.n
    rs, _ = oracle.preprocess(og, C, T, EPS)
    a = oracle.alpha(C, S, T)
    e_nb, e_st, e_tpa, rec = [], [], [], []
    for s in seeds:
        q = np.zeros(n)
        q[s] = 1.0
        fam, _ = oracle.cpi(og, q, C, EPS, 0, S - 1)
        nb = oracle.cpi(og, q, C, EPS, S, T - 1)[0] if T > S else np.zeros(n)
        st, _ = oracle.cpi(og, q, C, EPS, T, None)
        exact = fam + nb + st
        r = oracle.query(og, int(s), C, S, T, rs, EPS)
        e_nb.append(np.abs(nb - a * fam).sum())
        e_st.append(np.abs(st - rs).sum())
        e_tpa.append(np.abs(exact - r).sum())
        rec.append(len(np.intersect1d(np.argsort(-exact)[:k], np.argsort(-r)[:k])) / k)
    return np.mean(e_nb), np.mean(e_st), np.mean(e_tpa), np.mean(rec)


@pytest.mark.parametrize("S,T", SETTINGS)
def test_study_against_bounds_and_oracle(rmat14, S, T):
    import torch
    from paper_1708_02574_gb300 import accuracy
    t = tpa()
    seeds = torch.from_numpy(rmat14["seeds"]).cuda()
    row = accuracy.study(rmat14["g"], seeds, S, T, C, EPS, ks=(100,))
    b = accuracy.bounds(C, S, T)
    for part in ("neighbor", "stranger", "tpa"):
        assert row[part]["bound"] == pytest.approx(b[part])
        assert 0.0 <= row[part]["max"] <= b[part] + 1e-5, (part, row[part])
    # the parts add up to exact CPI
    fam, _ = t.cpi(rmat14["g"], seeds, C, EPS, 0, S - 1)
    st, _ = t.cpi(rmat14["g"], seeds, C, EPS, T, -1)
    nb = t.cpi(rmat14["g"], seeds, C, EPS, S, T - 1)[0] if T > S else torch.zeros_like(fam)
    exact, _ = t.cpi(rmat14["g"], seeds, C, EPS, 0, -1)
    assert float((fam.double() + nb.double() + st.double() - exact.double()).abs().sum(0).max()) <= 1e-5
    o_nb, o_st, o_tpa, o_rec = oracle_errors(rmat14["og"], rmat14["seeds"], S, T)
    assert abs(row["neighbor"]["error"] - o_nb) <= 2e-5
    assert abs(row["stranger"]["error"] - o_st) <= 2e-5
    assert abs(row["tpa"]["error"] - o_tpa) <= 2e-5
    assert 0.0 <= row["recall@100"] <= 1.0 and abs(row["recall@100"] - o_rec) <= 0.05


def test_sweep_shapes(rmat14):
    import torch
    from paper_1708_02574_gb300 import accuracy
    seeds = torch.from_numpy(rmat14["seeds"][:2]).cuda()
    res = accuracy.sweep(rmat14["g"], seeds, C, EPS, S_list=(2, 5), T_list=(4, 5, 10))
    assert [r["S"] for r in res["S_sweep"]] == [2, 5] and all(r["T"] == 10 for r in res["S_sweep"])
    assert [r["T"] for r in res["T_sweep"]] == [5, 10] and all(r["S"] == 5 for r in res["T_sweep"])
    # a larger S leaves less to approximate (Theorem 2's bound shrinks with S)
    assert res["S_sweep"][1]["tpa"]["bound"] < res["S_sweep"][0]["tpa"]["bound"]
