"""Pins for the FP64 adjoint oracle (gradient of a link-prediction loss on TPA scores).

The gradient is not in the paper; it is the chain rule through Algorithms 1-3
with A~ = w / rowsum.  It is pinned by:
  * central finite differences of the loss on edge weights w and on theta
    (w = exp(theta . f)),
  * a dense-matrix forward written here from the definitions,
  * the unweighted case (w = 1) reducing to the pinned TPA oracle,
and two planted mistakes in the adjoint must each be caught.
"""
import numpy as np
import pytest

import oracle
import synth

C, S, T = 0.15, 3, 5


def problem(kind="random", n=40, key=5, ntrip=6):
    n, s, d = synth.small_graph(kind, n, key=key)
    g = oracle.build_graph(n, s, d)
    rng = np.random.default_rng(key)
    cand = np.flatnonzero(g.outdeg > 0).astype(np.int32)
    seeds = rng.choice(cand, ntrip).astype(np.int32)
    pos = np.array([g.col_a[g.rp_a[x]] for x in seeds], np.int32)
    neg = rng.integers(0, n, ntrip).astype(np.int32)
    feat = rng.normal(size=(g.m, 4))
    theta = rng.normal(scale=0.3, size=4)
    return g, seeds, pos, neg, feat, theta


def dense_loss(g, w, seeds, pos, neg, K):
    n = g.n
    A = np.zeros((n, n))
    for u in range(n):
        for e in range(g.rp_a[u], g.rp_a[u + 1]):
            A[u, g.col_a[e]] = w[e]
    d = A.sum(axis=1)
    A[d > 0] /= d[d > 0, None]
    P = (1 - C) * A.T
    a = ((1 - C) ** S - (1 - C) ** T) / (1 - (1 - C) ** S)
    st = sum(np.linalg.matrix_power(P, i) @ np.full(n, C / n) for i in range(T, K + 1))
    L = 0.0
    for s, p, q in zip(seeds, pos, neg):
        e = np.zeros(n)
        e[s] = C
        fam = sum(np.linalg.matrix_power(P, i) @ e for i in range(S))
        r = (1 + a) * fam + st
        z = r[q] - r[p]
        L += np.log1p(np.exp(z))
    return L


def pin_fd_w():
    for kind in ("random", "random_nodead"):
        g, seeds, pos, neg, feat, theta = problem(kind)
        w = oracle.edge_weights(theta, feat)
        K = 12
        L, gw, _, _ = oracle.loss_grad(g, w, seeds, pos, neg, C, S, T, K)
        for e in np.linspace(0, g.m - 1, 9).astype(int):
            h = 1e-4 * w[e]                 # central differences: O(h^2) truncation, roundoff ~1e-12
            wp, wm = w.copy(), w.copy()
            wp[e] += h
            wm[e] -= h
            fd = (oracle.loss_grad(g, wp, seeds, pos, neg, C, S, T, K, want_grad=False)[0]
                  - oracle.loss_grad(g, wm, seeds, pos, neg, C, S, T, K, want_grad=False)[0]) / (2 * h)
            assert abs(fd - gw[e]) <= 1e-6 * abs(fd) + 1e-11, (kind, e, fd, gw[e])


def pin_fd_theta():
    g, seeds, pos, neg, feat, theta = problem("random", 50, key=9)
    K = 10
    w = oracle.edge_weights(theta, feat)
    _, gw, _, _ = oracle.loss_grad(g, w, seeds, pos, neg, C, S, T, K)
    gt = oracle.theta_grad(feat, w, gw)
    for j in range(theta.size):
        h = 1e-4
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (oracle.loss_grad(g, oracle.edge_weights(tp, feat), seeds, pos, neg, C, S, T, K, want_grad=False)[0]
              - oracle.loss_grad(g, oracle.edge_weights(tm, feat), seeds, pos, neg, C, S, T, K,
                                 want_grad=False)[0]) / (2 * h)
        assert abs(fd - gt[j]) <= 1e-6 * abs(fd) + 1e-10, (j, fd, gt[j])


def pin_dense_forward():
    g, seeds, pos, neg, feat, theta = problem("random", 30, key=2)
    w = oracle.edge_weights(theta, feat)
    K = 9
    L = oracle.loss_grad(g, w, seeds, pos, neg, C, S, T, K, want_grad=False)[0]
    assert abs(L - dense_loss(g, w, seeds, pos, neg, K)) < 1e-12


def pin_unweighted_is_tpa():
    """w = 1 gives A~ = 1/outdeg, and r_TPA at (pos, neg) equals the TPA oracle with K = its break index."""
    g, seeds, pos, neg, _, _ = problem("random_nodead", 64, key=4)
    rs, K = oracle.preprocess(g, C, T, 1e-9)
    va, vt, _ = oracle.weighted_vals(g, np.ones(g.m))
    assert np.allclose(va, g.val_a, rtol=0, atol=1e-15) and np.allclose(vt, g.val_t, rtol=0, atol=1e-15)
    _, _, rr, rstr = oracle.loss_grad(g, np.ones(g.m), seeds, pos, neg, C, S, T, K, want_grad=False)
    assert np.abs(rstr - rs).max() < 1e-15
    for t, s in enumerate(seeds):
        r = oracle.query(g, int(s), C, S, T, rs, 1e-9)
        assert abs(rr[t, 0] - r[pos[t]]) < 1e-15 and abs(rr[t, 1] - r[neg[t]]) < 1e-15


PINS = [pin_fd_w, pin_fd_theta, pin_dense_forward, pin_unweighted_is_tpa]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    oracle.set_adjoint_fault(0)
    pin()


@pytest.mark.parametrize("fault", [1, 2], ids=["no row-normalisation Jacobian", "stranger direct term dropped"])
def test_planted_adjoint_mistakes_are_caught(fault):
    caught = []
    try:
        oracle.set_adjoint_fault(fault)
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                caught.append(pin.__name__)
    finally:
        oracle.set_adjoint_fault(0)
    assert caught, fault
