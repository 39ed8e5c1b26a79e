"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

Nothing here computes any part of TPA or CPI: the module only draws counter-based
SplitMix64 random numbers (see ``synth.c``) and turns them into edge lists,
seed ids, batch sizes, edge features, parameter vectors and triples.

Recipes (the workloads stand in for the KONECT graphs of the paper's Table 2):

* ``rmat_edges(scale, edge_factor)``: R-MAT with (a, b, c, d) = (.57, .19, .19, .05),
  ``edge_factor * 2**scale`` raw edges, stream key 1.  Self-loops and duplicate
  edges are left in; dropping and merging them is the graph builder's job.
* ``query_seeds``: uniform over nodes that have an out-edge (stream key 2).
* ``batch_sizes``: sizes drawn uniformly from a set until a total is reached,
  last batch truncated (stream key 3).
* ``edge_features``: N(0, 1) float32 per edge and feature (stream key 4).
* ``theta``: N(0, 0.1^2) float32 (stream key 5).
* ``triples``: (seed, positive out-neighbour, uniform negative) (stream key 6).
* ``planted_edges(n, edge_factor, blocks, p_in)``: a planted-partition graph with
  communities, for the accuracy study (stream key 7).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

A, B, C, D = 0.57, 0.19, 0.19, 0.05


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` next to its source (host C, no GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, u64, i32p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        lib.synth_splitmix64.restype = u64
        lib.synth_splitmix64.argtypes = [u64, u64]
        lib.synth_uniform.restype = ctypes.c_double
        lib.synth_uniform.argtypes = [u64, u64]
        lib.synth_rmat.restype = ctypes.c_int
        lib.synth_rmat.argtypes = [ctypes.c_int, i64, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, u64, i32p, i32p, ctypes.c_int]
        lib.synth_planted.restype = ctypes.c_int
        lib.synth_planted.argtypes = [i64, i64, i64, ctypes.c_double, u64, i32p, i32p]
        lib.synth_has_out_edge.restype = None
        lib.synth_has_out_edge.argtypes = [i64, i64, i32p, i32p, i32p]
        lib.synth_pick_uniform.restype = None
        lib.synth_pick_uniform.argtypes = [i64, i32p, i64, u64, i32p]
        lib.synth_normal.restype = None
        lib.synth_normal.argtypes = [i64, u64, ctypes.c_double, ctypes.c_double, i32p]
        lib.synth_triples.restype = ctypes.c_int
        lib.synth_triples.argtypes = [i64, i64, i32p, i32p, i64, i32p, i64, u64, i32p, i32p, i32p]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def splitmix64(key: int, ctr: int) -> int:
    return int(_load().synth_splitmix64(key, ctr))


def uniform(key: int, ctr: int) -> float:
    return float(_load().synth_uniform(key, ctr))


def rmat_edges(scale: int, edge_factor: int = 16, a: float = A, b: float = B, c: float = C,
               key: int = 1, threads: int | None = None):
    """Raw R-MAT edge list (src, dst) as int32 arrays of length edge_factor * 2**scale."""
    m = int(edge_factor) << int(scale)
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    nt = threads or min(64, os.cpu_count() or 1)
    rc = _load().synth_rmat(int(scale), m, a, b, c, key, _ptr(src), _ptr(dst), nt)
    if rc != 0:
        raise ValueError("synth_rmat rejected its arguments")
    return src, dst


def planted_edges(n: int, edge_factor: int, blocks: int, p_in: float, key: int = 7):
    """Planted-partition graph (communities): ``edge_factor * n`` edges, uniform sources,
    destinations inside the source's block with probability ``p_in``, else uniform."""
    m = int(edge_factor) * int(n)
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    if _load().synth_planted(n, m, blocks, p_in, key, _ptr(src), _ptr(dst)) != 0:
        raise ValueError("synth_planted rejected its arguments")
    return src, dst


def nodes_with_out_edge(n: int, src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Sorted int32 ids of nodes that have at least one non-self-loop out-edge."""
    flag = np.empty(n, dtype=np.uint8)
    _load().synth_has_out_edge(n, src.size, _ptr(src), _ptr(dst), _ptr(flag))
    return np.flatnonzero(flag).astype(np.int32)


def query_seeds(candidates: np.ndarray, count: int, key: int = 2) -> np.ndarray:
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    if cand.size == 0:
        raise ValueError("no candidate seeds")
    out = np.empty(count, dtype=np.int32)
    _load().synth_pick_uniform(cand.size, _ptr(cand), count, key, _ptr(out))
    return out


def batch_sizes(total: int, choices=(1, 7, 32, 100, 256), key: int = 3) -> list[int]:
    """Sizes drawn uniformly from `choices` until `total` is reached (last one truncated)."""
    out, acc, i = [], 0, 0
    while acc < total:
        j = min(int(uniform(key, i) * len(choices)), len(choices) - 1)
        b = min(int(choices[j]), total - acc)
        out.append(b)
        acc += b
        i += 1
    return out


def normal(count: int, key: int, mean: float = 0.0, sd: float = 1.0) -> np.ndarray:
    out = np.empty(count, dtype=np.float32)
    _load().synth_normal(count, key, mean, sd, _ptr(out))
    return out


def edge_features(m: int, d: int = 8, key: int = 4) -> np.ndarray:
    return normal(m * d, key).reshape(m, d)


def theta(d: int = 8, key: int = 5) -> np.ndarray:
    return normal(d, key, 0.0, 0.1)


def triples(n: int, src: np.ndarray, dst: np.ndarray, candidates: np.ndarray, count: int,
            key: int = 6):
    cand = np.ascontiguousarray(candidates, dtype=np.int32)
    s = np.empty(count, dtype=np.int32)
    p = np.empty(count, dtype=np.int32)
    q = np.empty(count, dtype=np.int32)
    rc = _load().synth_triples(n, src.size, _ptr(src), _ptr(dst), cand.size, _ptr(cand), count,
                               key, _ptr(s), _ptr(p), _ptr(q))
    if rc != 0:
        raise MemoryError("synth_triples")
    return s, p, q


def small_graph(kind: str, n: int, key: int = 7):
    """Tiny named graphs used by tests: returns (n, src, dst) int32 arrays.

    kinds: 'cycle' (i -> i+1 mod n), 'star' (centre 0 <-> leaves 1..n-1),
    'complete' (all ordered pairs, no self-loops), 'random' (3n uniform pairs,
    self-loops and duplicates included), 'random_nodead' ('random' plus the
    cycle, so no node lacks an out-edge)."""
    if kind == "cycle":
        s = np.arange(n, dtype=np.int32)
        return n, s, ((s + 1) % n).astype(np.int32)
    if kind == "star":
        leaves = np.arange(1, n, dtype=np.int32)
        zero = np.zeros(n - 1, dtype=np.int32)
        return n, np.concatenate([zero, leaves]), np.concatenate([leaves, zero])
    if kind == "complete":
        s, t = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        keep = s != t
        return n, s[keep].astype(np.int32), t[keep].astype(np.int32)
    if kind in ("random", "random_nodead"):
        m = 3 * n
        u = np.array([uniform(key, i) for i in range(2 * m)])
        ids = np.minimum((u * n).astype(np.int64), n - 1).astype(np.int32)
        s, t = ids[:m], ids[m:]
        if kind == "random_nodead":
            c = np.arange(n, dtype=np.int32)
            s = np.concatenate([s, c])
            t = np.concatenate([t, (c + 1) % n]).astype(np.int32)
        return n, s.astype(np.int32), t.astype(np.int32)
    raise ValueError(kind)
