"""The scratch-free propagation step against the regular CPI entry point.

tpa_cpi_step_noalloc exists for callers that cannot allocate device memory
when they need a step (memory reserved by another allocator, or a loop that
must avoid cudaMalloc/cudaFree and their synchronisation); its scratch is a
fixed 16 MiB device array inside the library.  Here two calls in a row
(x0 -> x1 -> x2, accumulating r) must agree with tpa_cpi, which allocates its
own workspace, within the parity tolerance of the other GPU tests.  This file
sorts last so that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

C, EPS = 0.15, 1e-9
L1_TOL, MAX_TOL = 1e-5, 1e-7


def close(a, b, tag):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.abs(a - b)
    assert d.sum() <= L1_TOL and d.max() <= MAX_TOL, f"{tag}: L1 {d.sum():.3e} max-abs {d.max():.3e}"


def test_two_steps_match_cpi():
    import torch
    import paper_1708_02574_gb300 as tpa

    n = 1 << 14
    s, d = synth.rmat_edges(14, 16)
    g = tpa.build_graph(n, s, d)
    rp, col, val = tpa.get_csr(g, 0)
    m = g.m
    for seed in (0, int(synth.nodes_with_out_edge(n, s, d)[7])):
        x0 = torch.zeros(n, dtype=torch.float32, device="cuda")
        x0[seed] = C
        y1 = torch.empty(n, dtype=torch.float32, device="cuda")
        y2 = torch.empty(n, dtype=torch.float32, device="cuda")
        r = torch.zeros(n, dtype=torch.float32, device="cuda")
        l1 = torch.zeros(2, dtype=torch.float64, device="cuda")
        tpa.cpi_step_noalloc(n, m, rp, col, val, C, x0, y1, r, l1[0:1])
        tpa.cpi_step_noalloc(n, m, rp, col, val, C, y1, y2, r, l1[1:2])
        ref1 = tpa.cpi(g, [seed], C, EPS, 1, 1)[0][:, 0].cpu().numpy()
        ref2 = tpa.cpi(g, [seed], C, EPS, 2, 2)[0][:, 0].cpu().numpy()
        ref12 = tpa.cpi(g, [seed], C, EPS, 1, 2)[0][:, 0].cpu().numpy()
        close(y1.cpu().numpy(), ref1, f"x1 seed {seed}")
        close(y2.cpu().numpy(), ref2, f"x2 seed {seed}")
        close(r.cpu().numpy(), ref12, f"x1 + x2 seed {seed}")
        norms = l1.cpu().numpy()
        assert abs(norms[0] - ref1.astype(np.float64).sum()) <= 1e-6 * max(1.0, norms[0])
        assert abs(norms[1] - ref2.astype(np.float64).sum()) <= 1e-6 * max(1.0, norms[1])


def test_two_steps_match_the_oracle():
    """x1 = (1-c) A~^T x0 and x2 from two calls in a row, and r = x1 + x2,
    against the FP64 oracle's Algorithm 1 with s_iter = t_iter = 1, = 2 and
    s_iter = 1, t_iter = 2 (R-MAT scale 14 and a scale-16 graph that spans
    more merge-path tiles)."""
    import torch
    import oracle
    import paper_1708_02574_gb300 as tpa

    for scale in (14, 16):
        n = 1 << scale
        s, d = synth.rmat_edges(scale, 16)
        g = tpa.build_graph(n, s, d)
        og = oracle.build_graph(n, s, d)
        rp, col, val = tpa.get_csr(g, 0)
        m = g.m
        assert m == og.m
        cand = synth.nodes_with_out_edge(n, s, d)
        for seed in (int(cand[0]), int(cand[len(cand) // 2])):
            x0 = torch.zeros(n, dtype=torch.float32, device="cuda")
            x0[seed] = C
            y1 = torch.empty(n, dtype=torch.float32, device="cuda")
            y2 = torch.empty(n, dtype=torch.float32, device="cuda")
            r = torch.zeros(n, dtype=torch.float32, device="cuda")
            tpa.cpi_step_noalloc(n, m, rp, col, val, C, x0, y1, r)
            tpa.cpi_step_noalloc(n, m, rp, col, val, C, y1, y2, r)
            q = np.zeros(n)
            q[seed] = 1.0
            ref1, _ = oracle.cpi(og, q, C, EPS, 1, 1)
            ref2, _ = oracle.cpi(og, q, C, EPS, 2, 2)
            ref12, _ = oracle.cpi(og, q, C, EPS, 1, 2)
            close(y1.cpu().numpy(), ref1, f"x1 scale {scale} seed {seed}")
            close(y2.cpu().numpy(), ref2, f"x2 scale {scale} seed {seed}")
            close(r.cpu().numpy(), ref12, f"x1 + x2 scale {scale} seed {seed}")
        g.free()


def test_rejects_sizes_beyond_the_scratch():
    import paper_1708_02574_gb300 as tpa

    lib = tpa.library()
    st = lib.tpa_cpi_step_noalloc(ctypes.c_int64(150_000_000), ctypes.c_int64(1_000_000_000), None, None, None,
                                  ctypes.c_double(C), None, None, None, None, None)
    assert st == 1
    assert b"scratch" in lib.tpa_last_error()
    with pytest.raises(tpa.TpaError, match="EINVAL"):
        n = 8
        import torch
        rp = torch.zeros(n + 1, dtype=torch.int64)          # host memory is refused
        x = torch.zeros(n)
        tpa.cpi_step_noalloc(n, 0, rp, None, None, C, x, x)
