"""GPU adjoint (gradient of a link-prediction loss on TPA scores) against the FP64 oracle.

Workload: R-MAT scale 12 (4,096 nodes, edge factor 16), 8 features per edge ~ N(0,1)
(key 4), theta ~ N(0, 0.1^2) (key 5), w = exp(theta . f), triples (seed, out-neighbour,
uniform node) (key 6); c = 0.15, S = 5, T = 10.  Tolerances: weights and weighted
scores at FP32 parity; the FP32 gradient within 1e-3 relative (L2 norm of the error)
of the FP64 oracle gradient, and dL/dtheta within 1e-3 relative.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

C, S, T = 0.15, 5, 10


def tpa():
    import paper_1708_02574_gb300 as m
    return m


@pytest.fixture(scope="module")
def problem():
    import torch
    n = 1 << 12
    s, d = synth.rmat_edges(12, 16)
    og = oracle.build_graph(n, s, d)
    g = tpa().build_graph(n, s, d)
    feat = synth.edge_features(og.m, 8)
    theta = synth.theta(8)
    cand = synth.nodes_with_out_edge(n, s, d)
    seeds, pos, neg = synth.triples(n, s, d, cand, 48)
    return dict(n=n, og=og, g=g, feat=feat, theta=theta, seeds=seeds, pos=pos, neg=neg,
                feat_d=torch.from_numpy(feat).cuda(), theta_d=torch.from_numpy(theta).cuda())


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_edge_weights(problem):
    w = tpa().edge_weights(problem["feat_d"], problem["theta_d"]).cpu().numpy()
    ref = oracle.edge_weights(problem["theta"], problem["feat"])
    assert np.abs(w / ref - 1).max() < 1e-5


def test_weighted_query_parity(problem):
    """Weighted A~ in both CSR orders; preprocessing and queries on it match the oracle."""
    t = tpa()
    og, g = problem["og"], problem["g"]
    w = t.edge_weights(problem["feat_d"], problem["theta_d"])
    t.set_edge_weights(g, w)
    wd = oracle.edge_weights(problem["theta"], problem["feat"])
    va, vt, _ = oracle.weighted_vals(og, wd)
    _, col, val = t.get_csr(g, 0)
    assert np.abs(val.cpu().numpy() - vt).max() < 1e-6
    t.preprocess(g, C, T, 1e-9)
    rs_g, it = t.get_stranger(g)
    rs, rit = oracle.preprocess(og, C, T, 1e-9, val=vt)
    d = np.abs(rs_g.cpu().numpy() - rs)
    assert d.sum() <= 1e-5 and d.max() <= 1e-7 and abs(it - rit) <= 1
    seeds = problem["seeds"][:6]
    out = t.query(g, seeds, S).cpu().numpy()
    for j, sd in enumerate(seeds):
        ref = oracle.query(og, int(sd), C, S, T, rs, 1e-9, val=vt)
        d = np.abs(out[:, j] - ref)
        assert d.sum() <= 1e-5 and d.max() <= 1e-7, (j, d.sum(), d.max())


@pytest.mark.parametrize("ntrip,K", [(48, 24), (5, 10)])
def test_loss_grad_matches_oracle(problem, ntrip, K):
    t = tpa()
    og, g = problem["og"], problem["g"]
    w = t.edge_weights(problem["feat_d"], problem["theta_d"])
    t.set_edge_weights(g, w)
    sl = slice(0, ntrip)
    loss, gw = t.loss_grad(g, problem["seeds"][sl], problem["pos"][sl], problem["neg"][sl], C, S, T, K)
    wd = oracle.edge_weights(problem["theta"], problem["feat"])
    rloss, rgw, _, _ = oracle.loss_grad(og, wd, problem["seeds"][sl], problem["pos"][sl], problem["neg"][sl],
                                        C, S, T, K)
    assert abs(loss - rloss) <= 1e-5 * abs(rloss)
    gw = gw.cpu().numpy()
    assert rel(gw, rgw) < 1e-3, rel(gw, rgw)
    gth = t.theta_grad(problem["feat_d"], w, t.loss_grad(g, problem["seeds"][sl], problem["pos"][sl],
                                                         problem["neg"][sl], C, S, T, K)[1]).cpu().numpy()
    rgth = oracle.theta_grad(problem["feat"], wd, rgw)
    assert rel(gth, rgth) < 1e-3, (gth, rgth)


@pytest.mark.parametrize("width", [8, 16, 32])
def test_family_batch_widths(problem, width):
    """Family chains in batches of 8, 16 or 32 triples (48 triples: 6, 3 or 2
    batches, the last one of 32 partly padding) give the oracle's loss and
    gradient; widths differ from one another only by FP32 rounding."""
    t = tpa()
    og, g = problem["og"], problem["g"]
    w = t.edge_weights(problem["feat_d"], problem["theta_d"])
    t.set_edge_weights(g, w)
    K = 24
    t.set_adjoint_batch_width(width)
    try:
        assert t.get_adjoint_batch_width() == width
        loss, gw = t.loss_grad(g, problem["seeds"], problem["pos"], problem["neg"], C, S, T, K)
    finally:
        t.set_adjoint_batch_width(0)
    loss8, gw8 = t.loss_grad(g, problem["seeds"], problem["pos"], problem["neg"], C, S, T, K)
    wd = oracle.edge_weights(problem["theta"], problem["feat"])
    rloss, rgw, _, _ = oracle.loss_grad(og, wd, problem["seeds"], problem["pos"], problem["neg"], C, S, T, K)
    assert abs(loss - rloss) <= 1e-5 * abs(rloss)
    assert rel(gw.cpu().numpy(), rgw) < 1e-3
    assert rel(gw.cpu().numpy(), gw8.cpu().numpy()) < 1e-5
    with pytest.raises(t.TpaError, match="EINVAL"):
        t.set_adjoint_batch_width(12)


def test_autograd_function(problem):
    import torch
    t = tpa()
    theta = problem["theta_d"].clone().requires_grad_(True)
    K = 24
    loss = t.TPALinkLoss.apply(theta, problem["feat_d"], problem["g"], problem["seeds"], problem["pos"],
                               problem["neg"], C, S, T, K)
    loss.backward()
    wd = oracle.edge_weights(problem["theta"], problem["feat"])
    rloss, rgw, _, _ = oracle.loss_grad(problem["og"], wd, problem["seeds"], problem["pos"], problem["neg"],
                                        C, S, T, K)
    rgth = oracle.theta_grad(problem["feat"], wd, rgw)
    assert abs(loss.item() - rloss) <= 1e-5 * abs(rloss)
    assert rel(theta.grad.cpu().numpy(), rgth) < 1e-3
    # one gradient step lowers the loss
    with torch.no_grad():
        theta2 = theta - 5.0 * theta.grad / theta.grad.norm()
    loss2 = t.TPALinkLoss.apply(theta2, problem["feat_d"], problem["g"], problem["seeds"], problem["pos"],
                                problem["neg"], C, S, T, K)
    assert loss2.item() < loss.item()


def test_unit_weights_keep_preprocessing(problem):
    """The loss on an unweighted graph uses unit weights, which leave A~ bit-identical."""
    t = tpa()
    n, s, d = synth.small_graph("random_nodead", 500, key=3)
    g = t.build_graph(n, s, d)
    t.preprocess(g, C, T, 1e-9)
    _, _, v0 = t.get_csr(g, 1)
    loss, gw = t.loss_grad(g, [1, 2], [3, 4], [5, 6], C, S, T, 20)
    _, _, v1 = t.get_csr(g, 1)
    assert np.array_equal(v0.cpu().numpy(), v1.cpu().numpy())
    t.query(g, [1], S)    # still preprocessed


# ---------------------------------------------------------------------------
# Differentiation at full size: R-MAT scale 20 (1,048,576 nodes, 16,777,216 raw
# edges, key 1), 8 features per edge ~ N(0,1) (key 4), theta ~ N(0, 0.1^2)
# (key 5), 4,096 triples (key 6), K = 24 stranger steps.  The oracle computes
# the first 32 triples (the loss and its gradient are sums over triples, so a
# subset is a complete sample); the full 4,096-triple loss and gradient must
# equal the sum of four 1,024-triple parts (linearity holds at any size).

@pytest.fixture(scope="module")
def scale20():
    import torch
    n = 1 << 20
    s, d = synth.rmat_edges(20, 16)
    og = oracle.build_graph(n, s, d)
    g = tpa().build_graph(n, s, d)
    feat = synth.edge_features(og.m, 8)
    th = synth.theta(8)
    cand = synth.nodes_with_out_edge(n, s, d)
    seeds, pos, neg = synth.triples(n, s, d, cand, 4096)
    fd, td = torch.from_numpy(feat).cuda(), torch.from_numpy(th).cuda()
    w = tpa().edge_weights(fd, td)
    tpa().set_edge_weights(g, w)
    return dict(og=og, g=g, feat=feat, theta=th, fd=fd, w=w, seeds=seeds, pos=pos, neg=neg)


def test_scale20_loss_grad_sampled_triples(scale20):
    t = tpa()
    K, sl = 24, slice(0, 32)
    loss, gw = t.loss_grad(scale20["g"], scale20["seeds"][sl], scale20["pos"][sl], scale20["neg"][sl], C, S, T, K)
    wd = oracle.edge_weights(scale20["theta"], scale20["feat"])
    rloss, rgw, _, _ = oracle.loss_grad(scale20["og"], wd, scale20["seeds"][sl], scale20["pos"][sl],
                                        scale20["neg"][sl], C, S, T, K)
    assert abs(loss - rloss) <= 1e-5 * abs(rloss)
    assert rel(gw.cpu().numpy(), rgw) < 1e-3, rel(gw.cpu().numpy(), rgw)
    gth = t.theta_grad(scale20["fd"], scale20["w"], gw).cpu().numpy()
    assert rel(gth, oracle.theta_grad(scale20["feat"], wd, rgw)) < 1e-3


def test_scale20_loss_grad_is_a_sum_over_triples(scale20):
    import torch
    t = tpa()
    K = 24
    loss, gw = t.loss_grad(scale20["g"], scale20["seeds"], scale20["pos"], scale20["neg"], C, S, T, K)
    parts, gsum = 0.0, torch.zeros_like(gw, dtype=torch.float64)
    for q in range(4):
        sl = slice(1024 * q, 1024 * (q + 1))
        lq, gq = t.loss_grad(scale20["g"], scale20["seeds"][sl], scale20["pos"][sl], scale20["neg"][sl], C, S, T, K)
        parts += lq
        gsum += gq.double()
    assert np.isfinite(loss) and abs(loss - parts) <= 1e-6 * abs(parts)
    assert rel(gw.cpu().numpy(), gsum.cpu().numpy()) < 1e-5


# ---------------------------------------------------------------------------
# The stranger chain run for the count of the forward pass (the preprocessing
# break at eps = 1e-9, about 90-110 iterations), as TPALinkLoss(K=None) and
# the differentiation workload use it; iterate checkpointing; the loss alone.

def forward_K(t, g):
    t.preprocess(g, C, T, 1e-9)
    return max(int(t.get_stranger(g)[1]), T)


def test_loss_grad_at_forward_count(problem):
    t = tpa()
    og, g = problem["og"], problem["g"]
    w = t.edge_weights(problem["feat_d"], problem["theta_d"])
    t.set_edge_weights(g, w)
    K = forward_K(t, g)
    assert K > 60, K
    sl = slice(0, 48)
    loss, gw = t.loss_grad(g, problem["seeds"][sl], problem["pos"][sl], problem["neg"][sl], C, S, T, K)
    wd = oracle.edge_weights(problem["theta"], problem["feat"])
    rloss, rgw, _, _ = oracle.loss_grad(og, wd, problem["seeds"][sl], problem["pos"][sl], problem["neg"][sl],
                                        C, S, T, K)
    assert abs(loss - rloss) <= 1e-5 * abs(rloss)
    assert rel(gw.cpu().numpy(), rgw) < 1e-3, rel(gw.cpu().numpy(), rgw)
    gth = t.theta_grad(problem["feat_d"], w, gw).cpu().numpy()
    assert rel(gth, oracle.theta_grad(problem["feat"], wd, rgw)) < 1e-3


def test_checkpointed_iterates_are_bit_identical(problem):
    """With a budget too small for the K+1 iterates, the reverse sweep keeps
    every ceil(sqrt(K+1))-th one and recomputes the rest: same bits."""
    import torch
    t = tpa()
    g = problem["g"]
    w = t.edge_weights(problem["feat_d"], problem["theta_d"])
    t.set_edge_weights(g, w)
    K = forward_K(t, g)
    args = (problem["seeds"][:16], problem["pos"][:16], problem["neg"][:16], C, S, T, K)
    loss_a, gw_a = t.loss_grad(g, *args)
    try:
        t.set_adjoint_budget(1)
        loss_b, gw_b = t.loss_grad(g, *args)
    finally:
        t.set_adjoint_budget(16 << 30)
    assert loss_a == loss_b
    assert torch.equal(gw_a, gw_b)


def test_loss_alone_and_autograd_without_grad(problem):
    import torch
    t = tpa()
    g = problem["g"]
    w = t.edge_weights(problem["feat_d"], problem["theta_d"])
    t.set_edge_weights(g, w)
    K = 30
    args = (problem["seeds"], problem["pos"], problem["neg"], C, S, T, K)
    loss, _ = t.loss_grad(g, *args)
    loss_only, none = t.loss_grad(g, *args, want_grad=False)
    assert none is None and loss_only == loss
    theta = problem["theta_d"].clone()          # no gradient wanted: no reverse sweep
    with torch.no_grad():
        l2 = t.TPALinkLoss.apply(theta, problem["feat_d"], g, problem["seeds"], problem["pos"], problem["neg"],
                                 C, S, T, K)
    assert l2.item() == loss


def test_scale20_loss_grad_at_forward_count(scale20):
    """The differentiation workload's own K (the preprocessing count on the
    weighted R-MAT scale-20 graph), 32 triples against the FP64 oracle."""
    t = tpa()
    g = scale20["g"]
    K = forward_K(t, g)
    sl = slice(0, 32)
    loss, gw = t.loss_grad(g, scale20["seeds"][sl], scale20["pos"][sl], scale20["neg"][sl], C, S, T, K)
    wd = oracle.edge_weights(scale20["theta"], scale20["feat"])
    rloss, rgw, _, _ = oracle.loss_grad(scale20["og"], wd, scale20["seeds"][sl], scale20["pos"][sl],
                                        scale20["neg"][sl], C, S, T, K)
    assert abs(loss - rloss) <= 1e-5 * abs(rloss)
    assert rel(gw.cpu().numpy(), rgw) < 1e-3, rel(gw.cpu().numpy(), rgw)
