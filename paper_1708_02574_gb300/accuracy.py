"""Accuracy of TPA's two approximations against exact CPI: the error study of
Table 3 and of the S and T sweeps of Section IV (effects of parameters), run
on the GPU path for synthetic graphs.

For a seed s, exact CPI (Algorithm 1, tpa_cpi with s_iter / t_iter) splits
into the family, neighbor and stranger parts of Section III:
  r_family   = x_0 + ... + x_{S-1},
  r_neighbor = x_S + ... + x_{T-1},
  r_stranger = x_T + x_{T+1} + ...
TPA replaces the last two by
  r~_neighbor = alpha r_family                 (Section III-B),
  r~_stranger = PageRank's iterations >= T     (Algorithm 2),
and returns r_TPA = (1 + alpha) r_family + r~_stranger (Algorithm 3).  The
study reports, averaged over the seeds, the L1 errors
  ||r_neighbor - r~_neighbor||_1   against 2(1-c)^S - 2(1-c)^T (Lemma 3),
  ||r_stranger - r~_stranger||_1   against 2(1-c)^T          (Lemma 1),
  ||r_CPI - r_TPA||_1              against 2(1-c)^S          (Theorem 2),
each error's ratio to its bound (the percentage columns of Table 3), and
recall@k of r_TPA's top k against exact CPI's top k (Section IV accuracy).
Exact CPI runs to the preprocessing eps, so it holds iterations up to the
first x_i with ||x_i||_1 < eps.  Sums and norms are taken in FP64 over the
FP32 vectors.
"""
from __future__ import annotations

import time

from . import tpa as _t


def bounds(c: float, S: int, T: int) -> dict:
    return {"neighbor": 2 * (1 - c) ** S - 2 * (1 - c) ** T, "stranger": 2 * (1 - c) ** T,
            "tpa": 2 * (1 - c) ** S}


def _recall(exact, approx, k: int) -> float:
    """Mean over columns of |top-k(approx) & top-k(exact)| / k."""
    torch = _t._torch()
    k = min(k, exact.shape[0])
    te = torch.topk(exact, k, dim=0).indices
    ta = torch.topk(approx, k, dim=0).indices
    hits = 0
    for j in range(exact.shape[1]):
        hits += torch.isin(ta[:, j], te[:, j]).sum().item()
    return hits / (k * exact.shape[1])


def study(g, seeds, S: int, T: int, c: float = 0.15, eps: float = 1e-9, ks=(100,), preprocess: bool = True) -> dict:
    """Errors of one (S, T) for the given seeds (runs tpa_preprocess(c, T, eps)
    first unless preprocess is False and the graph already holds that T)."""
    torch = _t._torch()
    if not (1 <= S <= T):
        raise ValueError("need 1 <= S <= T")
    if preprocess:
        _t.preprocess(g, c, T, eps)
    alpha = ((1 - c) ** S - (1 - c) ** T) / (1 - (1 - c) ** S)
    fam, _ = _t.cpi(g, seeds, c, eps, 0, S - 1)
    st, _ = _t.cpi(g, seeds, c, eps, T, -1)
    fam, st = fam.double(), st.double()
    if T > S:
        nb = _t.cpi(g, seeds, c, eps, S, T - 1)[0].double()
    else:
        nb = torch.zeros_like(fam)
    exact = fam + nb + st
    r_st, _ = _t.get_stranger(g)
    r_st = r_st.double()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r_tpa = _t.query(g, seeds, S)
    torch.cuda.synchronize()
    online = time.perf_counter() - t0
    r_tpa = r_tpa.double()
    e_nb = (nb - alpha * fam).abs().sum(0)
    e_st = (st - r_st[:, None]).abs().sum(0)
    e_tpa = (exact - r_tpa).abs().sum(0)
    b = bounds(c, S, T)
    row = {"S": S, "T": T, "alpha": alpha, "seeds": len(seeds),
           "neighbor": {"error": e_nb.mean().item(), "max": e_nb.max().item(), "bound": b["neighbor"]},
           "stranger": {"error": e_st.mean().item(), "max": e_st.max().item(), "bound": b["stranger"]},
           "tpa": {"error": e_tpa.mean().item(), "max": e_tpa.max().item(), "bound": b["tpa"]},
           "online_ms_per_seed": 1e3 * online / len(seeds)}
    for part in ("neighbor", "stranger", "tpa"):
        row[part]["ratio"] = row[part]["error"] / row[part]["bound"] if row[part]["bound"] > 0 else 0.0
    for k in ks:
        row[f"recall@{k}"] = _recall(exact.float(), r_tpa.float(), k)
    return row


def sweep(g, seeds, c: float = 0.15, eps: float = 1e-9, S_fixed: int = 5, T_fixed: int = 10,
          S_list=range(2, 9), T_list=range(6, 21), ks=(100,)) -> dict:
    """The S sweep at T = T_fixed and the T sweep at S = S_fixed."""
    by_S = []
    _t.preprocess(g, c, T_fixed, eps)
    for S in S_list:
        by_S.append(study(g, seeds, S, T_fixed, c, eps, ks, preprocess=False))
    by_T = [study(g, seeds, S_fixed, T, c, eps, ks) for T in T_list if T >= S_fixed]
    _t.preprocess(g, c, T_fixed, eps)
    return {"S_sweep": by_S, "T_sweep": by_T}
