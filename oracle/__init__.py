"""FP64 CPU oracle for TPA (arXiv 1708.02574) -- TEST INFRASTRUCTURE ONLY.

Thin numpy/ctypes wrapper over ``tpa_oracle.c``.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package; the product path (``paper_1708_02574_gb300``) never does.

Functions follow the paper:
    build      -- Table 1: simple graph, row-normalised A~, CSR of A~^T and A~
    cpi        -- Algorithm 1 (Section II-C)
    preprocess -- Algorithm 2
    query      -- Algorithm 3 with the closed-form scale of Section III-B
    cpi_exact  -- Algorithm 1 with s_iter = 0, t_iter = infinity
    alpha      -- ((1-c)^S - (1-c)^T) / (1 - (1-c)^S)   (Section III-B, Lemma 2)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "tpa_oracle.c"), os.path.join(_HERE, "tpa_adjoint_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (plain C, -O2, no fast-math; OpenMP over independent rows)."""
    srcs = [s for s in _SRCS if os.path.exists(s)]
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in srcs)
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
                               "-shared", "-fPIC", *srcs, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, i64, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        lib.orc_set_fault.argtypes = [ctypes.c_int]
        lib.orc_set_fault.restype = None
        lib.orc_get_fault.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = None
        lib.orc_build.restype = i64
        lib.orc_build.argtypes = [i64, i64, P, P, P, P, P, P, P, P, P]
        lib.orc_cpi.restype = i64
        lib.orc_cpi.argtypes = [i64, P, P, P, P, f64, f64, i64, i64, P, P, i64]
        lib.orc_alpha.restype = f64
        lib.orc_alpha.argtypes = [f64, i64, i64]
        lib.orc_preprocess.restype = i64
        lib.orc_preprocess.argtypes = [i64, P, P, P, f64, f64, i64, P]
        lib.orc_query.restype = i64
        lib.orc_query.argtypes = [i64, P, P, P, f64, f64, i64, i64, ctypes.c_int32, P, P, P]
        lib.orc_cpi_exact.restype = i64
        lib.orc_cpi_exact.argtypes = [i64, P, P, P, f64, f64, ctypes.c_int32, P]
        lib.orc_query_set.restype = i64
        lib.orc_query_set.argtypes = [i64, P, P, P, f64, f64, i64, i64, i64, P, P, P]
        if hasattr(lib, "orc_adjoint_grad"):
            _bind_adjoint(lib)
        _lib = lib
    return _lib


def _bind_adjoint(lib):
    P, i64, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    lib.orc_adj_set_fault.argtypes = [ctypes.c_int]
    lib.orc_adj_set_fault.restype = None
    lib.orc_weighted_csr.restype = ctypes.c_int
    lib.orc_weighted_csr.argtypes = [i64, P, P, P, P, i64, P, P, P]
    lib.orc_adjoint_grad.restype = f64
    lib.orc_adjoint_grad.argtypes = [i64, i64, P, P, P, P, P, f64, i64, i64, i64, i64, P, P, P, P, P, P, P]


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def set_threads(t: int) -> None:
    """Threads of the oracle's loops over rows (0 = all cores); results do not depend on it."""
    _load().orc_set_threads(int(t))


def set_fault(k: int) -> None:
    """Plant mistake k in the oracle (0 = none).  For pin-strength tests only."""
    _load().orc_set_fault(int(k))


@dataclass
class Graph:
    n: int
    m: int
    rp_t: np.ndarray   # int64[n+1]  CSR(A~^T) row pointers (rows = destinations)
    col_t: np.ndarray  # int32[m]    sources, ascending within a row
    val_t: np.ndarray  # float64[m]  1/outdeg(source)
    rp_a: np.ndarray   # int64[n+1]  CSR(A~) row pointers (rows = sources)
    col_a: np.ndarray  # int32[m]    destinations, ascending within a row
    val_a: np.ndarray  # float64[m]
    outdeg: np.ndarray  # int32[n]


def build_graph(n: int, src: np.ndarray, dst: np.ndarray, with_a: bool = True) -> Graph:
    """orc_build: both CSRs of A~ (with_a=False: CSR(A~^T) alone, the CSR(A~)
    fields then None -- enough for Algorithms 1-3 on very large graphs)."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    mi = src.size
    rp_t = np.empty(n + 1, np.int64); col_t = np.empty(max(mi, 1), np.int32); val_t = np.empty(max(mi, 1))
    rp_a = col_a = val_a = None
    if with_a:
        rp_a = np.empty(n + 1, np.int64); col_a = np.empty(max(mi, 1), np.int32); val_a = np.empty(max(mi, 1))
    outdeg = np.empty(n, np.int32)
    m = lib.orc_build(n, mi, _p(src), _p(dst), _p(rp_t), _p(col_t), _p(val_t),
                      _p(rp_a), _p(col_a), _p(val_a), _p(outdeg))
    if m < 0:
        raise ValueError("orc_build rejected the edge list")
    return Graph(n, int(m), rp_t, col_t[:m], val_t[:m], rp_a, None if col_a is None else col_a[:m],
                 None if val_a is None else val_a[:m], outdeg)


def cpi(g: Graph, q: np.ndarray, c: float, eps: float, s_iter: int, t_iter: int | None,
        want_norms: bool = False, rp=None, col=None, val=None):
    """Algorithm 1.  Returns (r, iters[, norms]).  t_iter=None means infinity.

    rp/col/val override the unweighted CSR(A~^T) (used with weighted graphs)."""
    lib = _load()
    q = np.ascontiguousarray(q, dtype=np.float64)
    r = np.empty(g.n)
    cap = 100000 if want_norms else 0
    norms = np.zeros(cap) if want_norms else None
    it = lib.orc_cpi(g.n, _p(g.rp_t if rp is None else rp), _p(g.col_t if col is None else col),
                     _p(g.val_t if val is None else val), _p(q), c, eps, s_iter,
                     -1 if t_iter is None else t_iter, _p(r), _p(norms), cap)
    if it < 0:
        raise ValueError("orc_cpi rejected its arguments")
    if want_norms:
        return r, int(it), norms[: min(int(it), cap)]
    return r, int(it)


def alpha(c: float, S: int, T: int) -> float:
    return float(_load().orc_alpha(c, S, T))


def preprocess(g: Graph, c: float, T: int, eps: float = 1e-9, val=None):
    r = np.empty(g.n)
    it = _load().orc_preprocess(g.n, _p(g.rp_t), _p(g.col_t), _p(g.val_t if val is None else val),
                                c, eps, T, _p(r))
    if it < 0:
        raise ValueError("orc_preprocess")
    return r, int(it)


def query(g: Graph, seed: int, c: float, S: int, T: int, r_stranger: np.ndarray,
          eps: float = 1e-9, want_family: bool = False, val=None):
    out = np.empty(g.n)
    fam = np.empty(g.n) if want_family else None
    rs = np.ascontiguousarray(r_stranger, dtype=np.float64)
    it = _load().orc_query(g.n, _p(g.rp_t), _p(g.col_t), _p(g.val_t if val is None else val),
                           c, eps, S, T, int(seed), _p(rs), _p(out), _p(fam))
    if it < 0:
        raise ValueError("orc_query")
    return (out, fam) if want_family else out


def query_set(g: Graph, members, c: float, S: int, T: int, r_stranger: np.ndarray, eps: float = 1e-9):
    """Algorithm 3 for a seed set: q = 1/|S| on each listed member (a repeated member counts again)."""
    mem = np.ascontiguousarray(members, dtype=np.int32)
    out = np.empty(g.n)
    rs = np.ascontiguousarray(r_stranger, dtype=np.float64)
    it = _load().orc_query_set(g.n, _p(g.rp_t), _p(g.col_t), _p(g.val_t), c, eps, S, T, mem.size, _p(mem),
                               _p(rs), _p(out))
    if it < 0:
        raise ValueError("orc_query_set")
    return out


def cpi_exact(g: Graph, seed: int, c: float, eps: float = 1e-9):
    out = np.empty(g.n)
    it = _load().orc_cpi_exact(g.n, _p(g.rp_t), _p(g.col_t), _p(g.val_t), c, eps, int(seed), _p(out))
    if it < 0:
        raise ValueError("orc_cpi_exact")
    return out, int(it)


# ------------------------------------------------------------- adjoint ---
def set_adjoint_fault(k: int) -> None:
    """Plant mistake k in the adjoint oracle (0 = none).  For pin-strength tests only."""
    _load().orc_adj_set_fault(int(k))


def edge_weights(theta: np.ndarray, feat: np.ndarray) -> np.ndarray:
    """w_e = exp(theta . f_e) in FP64 (feat rows in CSR(A~) edge order)."""
    return np.exp(np.asarray(feat, dtype=np.float64) @ np.asarray(theta, dtype=np.float64))


def weighted_vals(g: Graph, w: np.ndarray):
    """(val_a, val_t, pos_t): A~ = w / rowsum in both CSR orders; pos_t maps CSR(A~) -> CSR(A~^T) positions."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    va = np.empty(max(g.m, 1))
    vt = np.empty(max(g.m, 1))
    pt = np.empty(max(g.m, 1), dtype=np.int64)
    rc = _load().orc_weighted_csr(g.n, _p(g.rp_a), _p(g.col_a), _p(w), _p(g.rp_t), g.m, _p(va), _p(vt), _p(pt))
    if rc != 0:
        raise MemoryError("orc_weighted_csr")
    return va[:g.m], vt[:g.m], pt[:g.m]


def loss_grad(g: Graph, w: np.ndarray, seeds, pos, neg, c: float, S: int, T: int, K: int, want_grad: bool = True):
    """Link-prediction loss on TPA scores and dL/dw (CSR(A~) order), FP64.

    Returns (loss, grad_w or None, r_pairs [ntrip, 2] = (r[pos], r[neg]), r_stranger)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    s = np.ascontiguousarray(seeds, dtype=np.int32)
    p = np.ascontiguousarray(pos, dtype=np.int32)
    q = np.ascontiguousarray(neg, dtype=np.int32)
    gw = np.empty(max(g.m, 1)) if want_grad else None
    rr = np.empty(2 * len(s))
    rs = np.empty(g.n)
    loss = _load().orc_adjoint_grad(g.n, g.m, _p(g.rp_a), _p(g.col_a), _p(g.rp_t), _p(g.col_t), _p(w), c, S, T, K,
                                    len(s), _p(s), _p(p), _p(q), _p(gw), _p(rr), _p(rs), None)
    if not np.isfinite(loss):
        raise ValueError("orc_adjoint_grad rejected its arguments")
    return loss, (gw[:g.m] if want_grad else None), rr.reshape(-1, 2), rs


def theta_grad(feat: np.ndarray, w: np.ndarray, grad_w: np.ndarray) -> np.ndarray:
    """dL/dtheta = sum_e dL/dw_e * w_e * f_e (w = exp(theta . f))."""
    return (np.asarray(grad_w, dtype=np.float64) * np.asarray(w, dtype=np.float64)) @ np.asarray(feat, dtype=np.float64)
