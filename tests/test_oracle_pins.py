"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each ``pin_*`` function raises AssertionError when the oracle disagrees with:
  * brute-force construction of the row-normalised adjacency (Table 1),
  * a dense LU solve of the RWR equation r = (1-c) A~^T r + c q (Section II-B,
    Theorem 1) and of PageRank (Section II-A),
  * matrix-power closed forms of the TPA parts (Section III, Algorithms 2-3),
  * closed forms on the directed cycle and the bidirectional star,
  * the L1-mass identities of Lemma 2 and the iteration count of Lemma 4,
  * the error bounds of Lemma 1, Lemma 3 and Theorem 2,
  * the bound constants printed in Table 3 (tests/golden/table3_bounds.txt),
  * seed sets: matrix powers applied to q = 1/|S| and linearity in q.

``test_planted_mistakes_are_caught`` plants plausible mistakes in the oracle
(on the CPU) and checks that at least one pin fails for each of them.
"""
import os

import numpy as np
import pytest

import oracle
import synth

C = 0.15
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table3_bounds.txt")


# ---------------------------------------------------------------- helpers ---
def dense_A(n, src, dst):
    """Row-normalised adjacency of the simple graph, by nested loops."""
    A = np.zeros((n, n))
    for s, d in zip(src.tolist(), dst.tolist()):
        if s != d:
            A[s, d] = 1.0
    deg = A.sum(axis=1)
    for u in range(n):
        if deg[u] > 0:
            A[u, :] /= deg[u]
    return A


def dense_rwr(A, q, c):
    n = A.shape[0]
    return np.linalg.solve(np.eye(n) - (1 - c) * A.T, c * q)


def graphs():
    out = []
    for kind, n in (("random", 40), ("random", 97), ("random_nodead", 64), ("complete", 9)):
        out.append((kind,) + synth.small_graph(kind, n, key=11 + n))
    return out


# ------------------------------------------------------------------- pins ---
def pin_csr_bruteforce():
    for kind, n, s, d in graphs():
        g = oracle.build_graph(n, s, d)
        A = dense_A(n, s, d)
        pattern = A > 0
        assert g.m == int(pattern.sum()), kind
        assert np.array_equal(g.outdeg, pattern.sum(axis=1).astype(np.int32)), kind
        # CSR(A~^T): rows are destinations
        for v in range(n):
            us = np.flatnonzero(pattern[:, v])
            seg = slice(g.rp_t[v], g.rp_t[v + 1])
            assert np.array_equal(g.col_t[seg], us), (kind, v)
            assert np.array_equal(g.val_t[seg], A[us, v]), (kind, v)
        # CSR(A~): rows are sources
        for u in range(n):
            vs = np.flatnonzero(pattern[u, :])
            seg = slice(g.rp_a[u], g.rp_a[u + 1])
            assert np.array_equal(g.col_a[seg], vs), (kind, u)
            assert np.array_equal(g.val_a[seg], A[u, vs]), (kind, u)


def pin_cpi_dense_solve():
    for kind, n, s, d in graphs():
        g = oracle.build_graph(n, s, d)
        A = dense_A(n, s, d)
        for seed in (0, n // 3, n - 1):
            q = np.zeros(n)
            q[seed] = 1.0
            r, _ = oracle.cpi(g, q, C, 1e-15, 0, None)
            ref = dense_rwr(A, q, C)
            assert np.abs(r - ref).sum() < 1e-12, (kind, seed, np.abs(r - ref).sum())
        q = np.full(n, 1.0 / n)
        r, _ = oracle.cpi(g, q, C, 1e-15, 0, None)
        assert np.abs(r - dense_rwr(A, q, C)).sum() < 1e-12, kind


def pin_tpa_matrix_powers():
    """r_TPA = (1+alpha) sum_{i<S} c P^i e_s + P^T (I-P)^{-1} (c/n) 1, P = (1-c) A~^T."""
    for kind, n, s, d in graphs():
        g = oracle.build_graph(n, s, d)
        A = dense_A(n, s, d)
        P = (1 - C) * A.T
        for S, T in ((5, 10), (2, 3), (4, 20), (1, 1)):
            rs, _ = oracle.preprocess(g, C, T, eps=1e-15)
            pr = np.linalg.solve(np.eye(n) - P, np.full(n, C / n))
            st = np.linalg.matrix_power(P, T) @ pr
            assert np.abs(rs - st).sum() < 1e-12, (kind, S, T)
            a = ((1 - C) ** S - (1 - C) ** T) / (1 - (1 - C) ** S)
            for seed in (1, n // 2):
                e = np.zeros(n)
                e[seed] = 1.0
                fam = sum(C * np.linalg.matrix_power(P, i) @ e for i in range(S))
                out, f = oracle.query(g, seed, C, S, T, rs, eps=1e-15, want_family=True)
                assert np.abs(f - fam).sum() < 1e-13, (kind, S, T, seed)
                assert np.abs(out - ((1 + a) * fam + st)).sum() < 1e-12, (kind, S, T, seed)


def pin_cycle_closed_form():
    n = 23
    _, s, d = synth.small_graph("cycle", n)
    g = oracle.build_graph(n, s, d)
    for seed in (0, 7):
        r, _ = oracle.cpi_exact(g, seed, C, eps=1e-15)
        dist = (np.arange(n) - seed) % n
        ref = C * (1 - C) ** dist / (1 - (1 - C) ** n)
        assert np.abs(r - ref).max() < 1e-14, seed
    q = np.full(n, 1.0 / n)
    p, _ = oracle.cpi(g, q, C, 1e-15, 0, None)
    assert np.abs(p - 1.0 / n).max() < 1e-14
    S, T = 5, 10
    rs, _ = oracle.preprocess(g, C, T, eps=1e-15)
    assert np.abs(rs - (1 - C) ** T / n).max() < 1e-14
    a = ((1 - C) ** S - (1 - C) ** T) / (1 - (1 - C) ** S)
    out = oracle.query(g, 4, C, S, T, rs, eps=1e-15)
    dist = (np.arange(n) - 4) % n
    fam = np.where(dist < S, C * (1 - C) ** dist, 0.0)
    assert np.abs(out - ((1 + a) * fam + (1 - C) ** T / n)).max() < 1e-14


def pin_star_closed_form():
    L = 12
    n, s, d = synth.small_graph("star", L + 1)
    g = oracle.build_graph(n, s, d)
    r, _ = oracle.cpi_exact(g, 0, C, eps=1e-15)
    den = 1 - (1 - C) ** 2
    assert abs(r[0] - C / den) < 1e-14
    assert np.abs(r[1:] - C * (1 - C) / (den * L)).max() < 1e-14
    # PageRank on the star: p0 = c/n + (1-c)(1-p0), leaves share the rest equally
    q = np.full(n, 1.0 / n)
    p, _ = oracle.cpi(g, q, C, 1e-15, 0, None)
    p0 = (C / n + (1 - C)) / (2 - C)
    assert abs(p[0] - p0) < 1e-14
    assert np.abs(p[1:] - (1 - p0) / L).max() < 1e-14


def pin_lemma2_mass():
    """Lemma 2 on graphs without deadends: ||x_i||_1 = c(1-c)^i, family and neighbour mass."""
    for kind in ("random_nodead", "complete", "cycle"):
        n, s, d = synth.small_graph(kind, 31, key=5)
        g = oracle.build_graph(n, s, d)
        assert (g.outdeg > 0).all()
        q = np.zeros(n)
        q[3] = 1.0
        r, it, norms = oracle.cpi(g, q, C, 1e-9, 0, None, want_norms=True)
        i = np.arange(1, it + 1)
        assert np.abs(norms - C * (1 - C) ** i).max() < 1e-15, kind
        # Lemma 4: the break comes at the first i with c(1-c)^i < eps
        assert it == 116, (kind, it)
        # r_CPI holds x_0 .. x_116
        assert abs(r.sum() - (1 - (1 - C) ** 117)) < 1e-13, kind
        for S, T in ((5, 10), (3, 7)):
            fam, _ = oracle.cpi(g, q, C, 1e-9, 0, S - 1)
            nb, _ = oracle.cpi(g, q, C, 1e-9, S, T - 1)
            assert abs(fam.sum() - (1 - (1 - C) ** S)) < 1e-14, kind
            assert abs(nb.sum() - ((1 - C) ** S - (1 - C) ** T)) < 1e-14, kind


def pin_bounds():
    """Lemma 1, Lemma 3 and Theorem 2 on graphs with and without deadends, and on
    planted-partition graphs (communities)."""
    planted = []
    for blocks, p_in in ((4, 0.9), (12, 0.6)):
        n = 96
        s, d = synth.planted_edges(n, 3, blocks, p_in, key=60 + blocks)
        planted.append((f"planted{blocks}", n, s, d))
    for kind, n, s, d in graphs() + planted:
        g = oracle.build_graph(n, s, d)
        for S, T in ((5, 10), (2, 4), (4, 6), (3, 3)):
            rs, _ = oracle.preprocess(g, C, T, eps=1e-13)
            for seed in range(0, n, max(1, n // 5)):
                q = np.zeros(n)
                q[seed] = 1.0
                exact, _ = oracle.cpi(g, q, C, 1e-13, 0, None)
                fam, _ = oracle.cpi(g, q, C, 1e-13, 0, S - 1)
                nb = oracle.cpi(g, q, C, 1e-13, S, T - 1)[0] if T > S else np.zeros(n)
                st, _ = oracle.cpi(g, q, C, 1e-13, T, None)
                tpa = oracle.query(g, seed, C, S, T, rs, eps=1e-13)
                a = oracle.alpha(C, S, T)
                tol = 1e-12
                assert np.abs(st - rs).sum() <= 2 * (1 - C) ** T + tol
                assert np.abs(nb - a * fam).sum() <= 2 * (1 - C) ** S - 2 * (1 - C) ** T + tol
                assert np.abs(exact - tpa).sum() <= 2 * (1 - C) ** S + tol
                # the three parts add up to exact CPI
                assert np.abs(fam + nb + st - exact).sum() < 1e-12


def pin_query_set():
    """Seed sets (q_s = 1/|S|, Section II-C): r_TPA from the matrix powers of
    P = (1-c) A~^T applied to that q, and the linearity of Algorithm 3 in q
    (the mean of the members' single-seed vectors, a repeated member counting
    twice)."""
    for kind, n, s, d in graphs():
        g = oracle.build_graph(n, s, d)
        P = (1 - C) * dense_A(n, s, d).T
        for S, T in ((5, 10), (2, 4)):
            rs, _ = oracle.preprocess(g, C, T, eps=1e-15)
            a = ((1 - C) ** S - (1 - C) ** T) / (1 - (1 - C) ** S)
            for members in ([3], [0, n - 1, n // 2], [5, 5, n - 2]):
                q = np.zeros(n)
                for v in members:
                    q[v] += 1.0 / len(members)
                fam = sum(C * np.linalg.matrix_power(P, i) @ q for i in range(S))
                got = oracle.query_set(g, members, C, S, T, rs, eps=1e-15)
                assert np.abs(got - ((1 + a) * fam + rs)).sum() < 1e-12, (kind, S, T, members)
                mean = sum(oracle.query(g, v, C, S, T, rs, eps=1e-15) for v in members) / len(members)
                assert np.abs(got - mean).sum() < 1e-12, (kind, S, T, members)


def read_table3():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, S, T, nb, st, tpa = line.split()
                rows.append((name, int(S), int(T), float(nb), float(st), float(tpa)))
    return rows


def pin_table3_constants():
    """Bound columns of Table 3, and alpha recovered from them (alpha = nb / (2 - tpa))."""
    rows = read_table3()
    assert len(rows) == 7
    for name, S, T, nb, st, tpa in rows:
        assert round(2 * (1 - C) ** S - 2 * (1 - C) ** T, 4) == nb, name
        assert round(2 * (1 - C) ** T, 4) == st, name
        assert round(2 * (1 - C) ** S, 4) == tpa, name
        a_printed = nb / (2 - tpa)
        # four printed decimals leave about 1e-4 of slack in the ratio
        assert abs(oracle.alpha(C, S, T) - a_printed) < 3e-4, name


PINS = [pin_csr_bruteforce, pin_cpi_dense_solve, pin_tpa_matrix_powers, pin_cycle_closed_form,
        pin_star_closed_form, pin_lemma2_mass, pin_bounds, pin_table3_constants, pin_query_set]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    oracle.set_fault(0)
    pin()


FAULTS = {1: "A~ instead of A~^T", 2: "x0 dropped from r", 3: "decay (1-c) dropped",
          4: "alpha sign flipped", 5: "t_iter exclusive", 6: "normalised by in-degree",
          7: "norm tested before adding x_i", 8: "PageRank q unnormalised", 9: "seed-set q unnormalised"}


@pytest.mark.parametrize("fault", sorted(FAULTS), ids=[FAULTS[k] for k in sorted(FAULTS)])
def test_planted_mistakes_are_caught(fault):
    caught = []
    try:
        oracle.set_fault(fault)
        for pin in PINS:
            try:
                pin()
            except (AssertionError, ValueError, np.linalg.LinAlgError):
                caught.append(pin.__name__)
    finally:
        oracle.set_fault(0)
    assert caught, f"no pin caught planted mistake {fault}: {FAULTS[fault]}"


def test_query_rejects_bad_input():
    n, s, d = synth.small_graph("cycle", 5)
    g = oracle.build_graph(n, s, d)
    rs, _ = oracle.preprocess(g, C, 10)
    with pytest.raises(ValueError):
        oracle.query(g, 5, C, 5, 10, rs)
    with pytest.raises(ValueError):
        oracle.query(g, 0, C, 6, 5, rs)


def test_oracle_threads_do_not_change_results():
    """The oracle's loops over rows may run on several threads; every row's
    sum keeps its order and norms are summed sequentially, so the CSR, the
    preprocessing vector and a query are bit-identical on 1 and on many
    threads (R-MAT scale 12 with duplicates and self-loops in the raw list)."""
    n = 1 << 12
    s, d = synth.rmat_edges(12, 16)
    outs = []
    try:
        for t in (1, 0, 3):
            oracle.set_threads(t)
            og = oracle.build_graph(n, s, d)
            rs, it = oracle.preprocess(og, 0.15, 10, 1e-9)
            q = oracle.query(og, 5, 0.15, 5, 10, rs, 1e-9)
            outs.append((og.rp_t.copy(), og.col_t.copy(), og.val_t.copy(), og.rp_a.copy(), og.col_a.copy(),
                         rs, it, q))
    finally:
        oracle.set_threads(0)
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a, b)
