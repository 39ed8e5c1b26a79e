"""ctypes binding of libtpa (names follow include/tpa.h without the ``tpa_`` prefix).

Arrays may be numpy arrays (host) or torch tensors (host or CUDA).  Results are
returned as CUDA torch tensors allocated on the current device, written on the
current torch stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

_lib = None

STATUS = {0: "TPA_OK", 1: "TPA_EINVAL", 2: "TPA_ENOMEM", 3: "TPA_ECUDA", 4: "TPA_ESTATE", 5: "TPA_ETIMEOUT"}


class TpaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def library():
    """Load libtpa.so (compiling it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or _build.stale():
        _build.build()
    lib = ctypes.CDLL(path)
    P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "tpa_last_error": (ctypes.c_char_p, []),
        "tpa_build_graph": (i32, [i64, i64, P, P, P, ctypes.POINTER(P)]),
        "tpa_free_graph": (None, [P]),
        "tpa_graph_info": (i32, [P, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "tpa_get_csr": (i32, [P, i32, P, P, P, P]),
        "tpa_preprocess": (i32, [P, f64, i32, f64, P]),
        "tpa_get_stranger": (i32, [P, P, ctypes.POINTER(i64), P]),
        "tpa_query": (i32, [P, P, i32, i32, P, P]),
        "tpa_query_sets": (i32, [P, P, P, i32, i32, P, P]),
        "tpa_cpi": (i32, [P, P, i32, f64, f64, i32, i32, P, P, P]),
        "tpa_cpi_exact": (i32, [P, ctypes.c_int32, f64, f64, P, P, P]),
        "tpa_save_preprocessed": (i32, [P, ctypes.c_char_p]),
        "tpa_load_preprocessed": (i32, [P, ctypes.c_char_p, P]),
        "tpa_cpi_step_noalloc": (i32, [i64, i64, P, P, P, f64, P, P, P, P, P]),
        "tpa_set_edge_weights": (i32, [P, P, P]),
        "tpa_edge_weights": (i32, [P, P, i32, i64, P, P]),
        "tpa_loss_grad": (i32, [P, P, P, P, i32, f64, i32, i32, i32, ctypes.POINTER(f64), P, P]),
        "tpa_theta_grad": (i32, [P, P, P, i32, i64, P, P]),
        "tpa_sync": (i32, [P, P]),
        "tpa_set_adjoint_budget": (i32, [ctypes.c_uint64]),
        "tpa_set_adjoint_batch_width": (i32, [i32]),
        "tpa_get_adjoint_batch_width": (i32, []),
        "tpa_server_sync": (i32, [P, P]),
        "tpa_server_create": (i32, [P, i32, i32, P, i64, P, ctypes.POINTER(P)]),
        "tpa_server_query": (i32, [P, P, i32, P]),
        "tpa_server_result": (i32, [P, ctypes.POINTER(P), ctypes.POINTER(i64)]),
        "tpa_server_stats": (i32, [P, i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                   ctypes.POINTER(i64)]),
        "tpa_server_free": (None, [P]),
        "tpa_launch_count": (ctypes.c_uint64, []),
        "tpa_variant_count": (i32, []),
        "tpa_variant_info": (i32, [i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                   ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "tpa_variant_name": (ctypes.c_char_p, [i32]),
        "tpa_get_variant": (i32, [i32]),
        "tpa_set_variant": (i32, [i32, i32]),
        "tpa_set_batch_width": (i32, [i32]),
        "tpa_get_batch_width": (i32, []),
        "tpa_set_cpi_batch_width": (i32, [i32]),
        "tpa_get_cpi_batch_width": (i32, []),
        "tpa_set_push": (i32, [i32]),
        "tpa_set_output_group_width": (i32, [i32]),
        "tpa_get_output_group_width": (i32, []),
        "tpa_set_pattern": (i32, [i32]),
        "tpa_seed_order": (i32, [P, i32, i32, P]),
        "tpa_profile_reset": (i32, [i32]),
        "tpa_profile_read": (i32, [P, i32, ctypes.POINTER(i32)]),
        "tpa_probe_gather": (i32, [P, i32, i32, P, ctypes.POINTER(f64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int):
    if st != 0:
        raise TpaError(st, library().tpa_last_error().decode(errors="replace"))


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(a):
    """Raw pointer of a contiguous numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(a.ctypes.data)
    assert a.is_contiguous()
    return ctypes.c_void_p(a.data_ptr())


def _as_i32(a):
    torch = _torch()
    if isinstance(a, torch.Tensor):
        return a.to(torch.int32).contiguous()
    return np.ascontiguousarray(a, dtype=np.int32)


class Graph:
    """Owner of a ``tpa_graph`` handle."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @property
    def handle(self):
        if not self._h:
            raise TpaError(1, "graph was freed")
        return self._h

    def free(self):
        if self._h:
            library().tpa_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def n(self) -> int:
        return graph_info(self)[0]

    @property
    def m(self) -> int:
        return graph_info(self)[1]


def build_graph(n: int, src, dst) -> Graph:
    """tpa_build_graph: row-normalised adjacency of the simple graph (Table 1)."""
    s, d = _as_i32(src), _as_i32(dst)
    h = ctypes.c_void_p()
    m = len(s)
    _check(library().tpa_build_graph(int(n), int(m), _ptr(s), _ptr(d), _stream(), ctypes.byref(h)))
    return Graph(h)


def graph_info(g: Graph):
    n, m = ctypes.c_int64(), ctypes.c_int64()
    _check(library().tpa_graph_info(g.handle, ctypes.byref(n), ctypes.byref(m)))
    return n.value, m.value


def get_csr(g: Graph, which: int = 0):
    """CSR of A~^T (which=0) or A~ (which=1) as CUDA tensors (row_ptr, col, val)."""
    torch = _torch()
    n, m = graph_info(g)
    rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(max(m, 1), dtype=torch.int32, device="cuda")
    val = torch.empty(max(m, 1), dtype=torch.float32, device="cuda")
    _check(library().tpa_get_csr(g.handle, int(which), _ptr(rp), _ptr(col), _ptr(val), _stream()))
    return rp, col[:m], val[:m]


def preprocess(g: Graph, c: float = 0.15, T: int = 10, eps: float = 1e-9) -> None:
    """tpa_preprocess (Algorithm 2)."""
    _check(library().tpa_preprocess(g.handle, float(c), int(T), float(eps), _stream()))


def get_stranger(g: Graph):
    torch = _torch()
    n, _ = graph_info(g)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    it = ctypes.c_int64()
    _check(library().tpa_get_stranger(g.handle, _ptr(out), ctypes.byref(it), _stream()))
    return out, it.value


def query(g: Graph, seeds, S: int = 5, out=None):
    """tpa_query (Algorithm 3) for k single-seed queries; returns float32 [n, k]."""
    torch = _torch()
    s = _as_i32(seeds)
    k = len(s)
    n, _ = graph_info(g)
    if out is None:
        out = torch.empty((n, k), dtype=torch.float32, device="cuda")
    _check(library().tpa_query(g.handle, _ptr(s), int(k), int(S), _ptr(out), _stream()))
    return out


def query_sets(g: Graph, sets, S: int = 5, out=None):
    """tpa_query_sets (Algorithm 3 with q = 1/|S| over each seed set); ``sets`` is a
    list of member lists.  Returns float32 [n, len(sets)]."""
    torch = _torch()
    sets = [list(x) for x in sets]
    ptr = np.zeros(len(sets) + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(x) for x in sets])
    mem = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.int64) for x in sets]) if sets else
                               np.zeros(0), dtype=np.int32)
    n, _ = graph_info(g)
    if out is None:
        out = torch.empty((n, len(sets)), dtype=torch.float32, device="cuda")
    _check(library().tpa_query_sets(g.handle, _ptr(ptr), _ptr(mem), int(len(sets)), int(S), _ptr(out), _stream()))
    return out


class Server:
    """tpa_server: request batches of up to max_k seeds answered by CUDA-graph
    replays.  Results land in ``out`` (a CUDA float32 tensor [n, max_k], the
    first k columns after a batch of k seeds); the graph must outlive it."""

    def __init__(self, g: Graph, S: int = 5, max_k: int = 256, out=None):
        torch = _torch()
        n, _ = graph_info(g)
        if out is None:
            out = torch.empty((n, max_k), dtype=torch.float32, device="cuda")
        assert out.dtype == torch.float32 and out.is_cuda and out.is_contiguous() and out.shape[0] == n
        self.g, self.out, self.max_k = g, out, int(max_k)
        self._h = ctypes.c_void_p()
        _check(library().tpa_server_create(g.handle, int(S), int(max_k), _ptr(out), int(out.shape[1]), _stream(),
                                           ctypes.byref(self._h)))

    def query(self, seeds):
        """Answer one batch; returns the [n, k] view of ``out`` holding its scores."""
        s = _as_i32(seeds)
        k = len(s)
        _check(library().tpa_server_query(self._h, _ptr(s), int(k), _stream()))
        return self.out[:, :k]

    def sync(self) -> None:
        """tpa_server_sync: wait for the server's work, failing if a bounded device wait gave up."""
        _check(library().tpa_server_sync(self._h, _stream()))

    def stats(self, k: int = 0) -> dict:
        gr, rp, lp, cp = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(library().tpa_server_stats(self._h, int(k), ctypes.byref(gr), ctypes.byref(rp), ctypes.byref(lp),
                                          ctypes.byref(cp)))
        return {"graphs": gr.value, "replays": rp.value, "launches_per_replay": lp.value, "captures": cp.value}

    def free(self):
        if self._h:
            library().tpa_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def cpi(g: Graph, seeds, c: float = 0.15, eps: float = 1e-9, s_iter: int = 0, t_iter: int = -1, out=None):
    """tpa_cpi (Algorithm 1) for k single-seed vectors; returns (float32 [n, k], int32 iters[k])."""
    torch = _torch()
    s = _as_i32(seeds)
    k = len(s)
    n, _ = graph_info(g)
    if out is None:
        out = torch.empty((n, k), dtype=torch.float32, device="cuda")
    iters = torch.empty(k, dtype=torch.int32, device="cuda")
    _check(library().tpa_cpi(g.handle, _ptr(s), int(k), float(c), float(eps), int(s_iter), int(t_iter),
                             _ptr(out), _ptr(iters), _stream()))
    return out, iters


def cpi_exact(g: Graph, seed: int, c: float = 0.15, eps: float = 1e-9):
    """tpa_cpi_exact: exact RWR by CPI for one seed; returns (float32 [n], iterations)."""
    torch = _torch()
    n, _ = graph_info(g)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    it = np.zeros(1, dtype=np.int32)
    _check(library().tpa_cpi_exact(g.handle, int(seed), float(c), float(eps), _ptr(out), _ptr(it), _stream()))
    return out, int(it[0])


def save_preprocessed(g: Graph, path: str) -> None:
    _check(library().tpa_save_preprocessed(g.handle, os.fsencode(path)))


def load_preprocessed(g: Graph, path: str) -> None:
    _check(library().tpa_load_preprocessed(g.handle, os.fsencode(path), _stream()))


class _KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("alg_bytes", ctypes.c_double)]


def launch_count() -> int:
    """Kernel launches issued by libtpa since it was loaded."""
    return int(library().tpa_launch_count())


def profile_reset(timing: bool = False) -> None:
    """Clear kernel statistics; with timing, bracket SpMV/SpMM and fixup launches with CUDA events."""
    _check(library().tpa_profile_reset(1 if timing else 0))


def probe_gather(g, kp: int, reps: int = 5) -> float:
    """tpa_probe_gather: ms per pass of the gather-only probe (kp = 1 or 8) over g's CSR(A~^T)."""
    ms = ctypes.c_double(0.0)
    _check(library().tpa_probe_gather(g.handle, int(kp), int(reps), _stream(), ctypes.byref(ms)))
    return ms.value


def profile_read() -> dict:
    """Per kernel family: launches, summed event time (ms) and algorithmic bytes."""
    cap = 64
    arr = (_KernelStat * cap)()
    cnt = ctypes.c_int()
    _check(library().tpa_profile_read(ctypes.cast(arr, ctypes.c_void_p), cap, ctypes.byref(cnt)))
    return {arr[i].name.decode(): dict(launches=int(arr[i].launches), total_ms=float(arr[i].total_ms),
                                       alg_bytes=float(arr[i].alg_bytes)) for i in range(min(cnt.value, cap))}


def variants() -> list[dict]:
    """Compiled SpMV/SpMM variants: padded width, lanes per walker, columns per lane, steps, threads, name."""
    lib = library()
    out = []
    for i in range(lib.tpa_variant_count()):
        v = [ctypes.c_int() for _ in range(5)]
        _check(lib.tpa_variant_info(i, *[ctypes.byref(x) for x in v]))
        out.append(dict(index=i, kp=v[0].value, lanes=v[1].value, cols_per_lane=v[2].value, items=v[3].value,
                        threads=v[4].value, name=lib.tpa_variant_name(i).decode()))
    return out


def get_variant(kp: int) -> int:
    """Index of the variant in effect for padded width kp (forced, else default)."""
    return int(library().tpa_get_variant(int(kp)))


def set_variant(kp: int, idx: int) -> None:
    _check(library().tpa_set_variant(int(kp), int(idx)))


def set_batch_width(width: int) -> None:
    _check(library().tpa_set_batch_width(int(width)))


def get_batch_width() -> int:
    return int(library().tpa_get_batch_width())


def set_cpi_batch_width(width: int) -> None:
    _check(library().tpa_set_cpi_batch_width(int(width)))


def get_cpi_batch_width() -> int:
    return int(library().tpa_get_cpi_batch_width())


def cpi_step_noalloc(n: int, m: int, row_ptr, col, val, c: float, x, y, r=None, l1=None) -> None:
    """tpa_cpi_step_noalloc: y = (1-c) A~^T x (and r += y, l1[0] = ||y||_1) with no allocation.

    All tensors must be CUDA tensors; the CSR is that of A~^T (rows = destinations)."""
    _check(library().tpa_cpi_step_noalloc(int(n), int(m), _ptr(row_ptr), _ptr(col), _ptr(val), float(c), _ptr(x),
                                          _ptr(y), _ptr(r), _ptr(l1), _stream()))


def set_output_group_width(width: int) -> None:
    """Column groups of a query into page-locked host memory: 0 automatic (default), -1 direct writes, else the width."""
    _check(library().tpa_set_output_group_width(int(width)))


def get_output_group_width() -> int:
    return int(library().tpa_get_output_group_width())


def set_push(enable: bool) -> None:
    """Push the sparse first family iterates of a query (default) or pull every iteration."""
    _check(library().tpa_set_push(1 if enable else 0))


def seed_order(outdeg, S: int = 5) -> np.ndarray:
    """tpa_seed_order: the order tpa_query runs seeds with these out-degrees in (host only)."""
    od = np.ascontiguousarray(outdeg, dtype=np.int32)
    perm = np.empty(od.size, dtype=np.int32)
    _check(library().tpa_seed_order(_ptr(od), int(od.size), int(S), _ptr(perm)))
    return perm


def set_pattern(enable: bool) -> None:
    """Pattern-only products on unweighted graphs (default: x kept scaled by 1/outdeg, no value
    array read) or products that read the value array."""
    _check(library().tpa_set_pattern(1 if enable else 0))


# ------------------------------------------------------------- gradients ---
def set_edge_weights(g: Graph, w) -> None:
    """tpa_set_edge_weights: A~ = w / rowsum (w in CSR(A~) edge order)."""
    w = w.contiguous() if not isinstance(w, np.ndarray) else np.ascontiguousarray(w, dtype=np.float32)
    _check(library().tpa_set_edge_weights(g.handle, _ptr(w), _stream()))


def edge_weights(feat, theta):
    """tpa_edge_weights: w_e = exp(theta . f_e) for CUDA tensors feat [m, d] and theta [d]."""
    torch = _torch()
    feat = feat.contiguous().to(torch.float32)
    theta = theta.contiguous().to(torch.float32)
    m, d = feat.shape
    w = torch.empty(m, dtype=torch.float32, device=feat.device)
    _check(library().tpa_edge_weights(_ptr(feat), _ptr(theta), int(d), int(m), _ptr(w), _stream()))
    return w


def loss_grad(g: Graph, seeds, pos, neg, c: float = 0.15, S: int = 5, T: int = 10, K: int = 100,
              want_grad: bool = True):
    """tpa_loss_grad: (loss, dL/dw as a CUDA float32 tensor in CSR(A~) order); with
    want_grad=False the loss alone (no reverse sweep) and None."""
    torch = _torch()
    s, p, q = _as_i32(seeds), _as_i32(pos), _as_i32(neg)
    n, m = graph_info(g)
    gw = torch.empty(max(m, 1), dtype=torch.float32, device="cuda") if want_grad else None
    loss = ctypes.c_double()
    _check(library().tpa_loss_grad(g.handle, _ptr(s), _ptr(p), _ptr(q), int(len(s)), float(c), int(S), int(T),
                                   int(K), ctypes.byref(loss), _ptr(gw), _stream()))
    return loss.value, (gw[:m] if want_grad else None)


def set_adjoint_budget(nbytes: int) -> None:
    """tpa_set_adjoint_budget: iterate bytes kept before checkpointing."""
    _check(library().tpa_set_adjoint_budget(int(nbytes)))


def set_adjoint_batch_width(width: int) -> None:
    """tpa_set_adjoint_batch_width: triples per family batch (8, 16, 32; 0 the default)."""
    _check(library().tpa_set_adjoint_batch_width(int(width)))


def get_adjoint_batch_width() -> int:
    return int(library().tpa_get_adjoint_batch_width())


def sync(g: Graph) -> None:
    """tpa_sync: wait for the graph's work; TpaError(TPA_ETIMEOUT) if a bounded device wait gave up."""
    _check(library().tpa_sync(g.handle, _stream()))


def theta_grad(feat, w, grad_w):
    """tpa_theta_grad: dL/dtheta (CUDA float64 tensor [d])."""
    torch = _torch()
    feat = feat.contiguous().to(torch.float32)
    m, d = feat.shape
    out = torch.empty(d, dtype=torch.float64, device=feat.device)
    _check(library().tpa_theta_grad(_ptr(feat), _ptr(w.contiguous()), _ptr(grad_w.contiguous()), int(d), int(m),
                                    _ptr(out), _stream()))
    return out
