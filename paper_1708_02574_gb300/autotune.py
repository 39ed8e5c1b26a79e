"""Autotuner for the SpMV/SpMM that runs every CPI iteration.

Two knobs are tuned on the graph at hand:
  * the batch width (seeds per CPI chunk, the right-hand-side tile width of the
    SpMM): narrow chunks keep the iterate block X[n][width] in L2 and let light
    seeds use the push path for x1 and x2, wide chunks reuse each streamed
    nonzero for more seeds;
  * the kernel variant per width (lanes per merge-path walker, columns per
    lane, path steps per lane), and the k = 1 variant of preprocessing.
Every candidate is timed with CUDA events on the current stream after a
warm-up call; the fastest is applied with tpa_set_variant/tpa_set_batch_width,
except that a library default within TIE of the fastest is kept (so the
choice does not flip between runs on timing noise).  Results differ between
candidates only by FP32 rounding order.
"""
from __future__ import annotations

import time

from . import tpa

TIE = 0.03   # relative margin within which a default wins


def pick_fastest(times: dict, default, tie: float = TIE):
    """Key of the smallest time in `times`, except that `default` (when timed)
    wins if it is within a factor (1 + tie) of that smallest time."""
    best = min(times, key=lambda k: times[k])
    if default in times and times[default] <= times[best] * (1.0 + tie):
        return default
    return best


def pick_query(results: list, defaults: dict, default_width: int, tie: float = TIE) -> dict:
    """The query setting with the highest throughput in `results` (dicts with
    width, variant, seeds_per_s), except that within a factor (1 + tie) of it
    the default variant of the best width wins, then the default width's
    default variant."""
    best = max(results, key=lambda r: r["seeds_per_s"])
    for cand in ([r for r in results if r["width"] == best["width"] and r["variant"] == defaults[best["width"]]] +
                 [r for r in results if r["width"] == default_width and r["variant"] == defaults[default_width]]):
        if cand["seeds_per_s"] >= best["seeds_per_s"] / (1.0 + tie):
            return cand
    return best


def _time(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / reps


def tune_preprocess(g: tpa.Graph, c: float, T: int, eps: float, reps: int = 1) -> dict:
    """Pick the fastest k = 1 variant by timing tpa_preprocess."""
    tpa.set_variant(1, -1)
    default = tpa.get_variant(1)
    times = {}
    for v in tpa.variants():
        if v["kp"] != 1:
            continue
        tpa.set_variant(1, v["index"])
        times[v["index"]] = _time(lambda: tpa.preprocess(g, c, T, eps), reps)
    best = pick_fastest(times, default)
    tpa.set_variant(1, best)
    tpa.preprocess(g, c, T, eps)
    return {"variant": best, "seconds": times[best]}


def tune_query(g: tpa.Graph, seeds, S: int, widths=(1, 2, 4, 8, 16, 32, 64, 128, 256), reps: int = 2,
               max_seeds: int = 256) -> dict:
    """Pick the batch width and variant with the highest query throughput on `seeds`."""
    import torch
    n = g.n
    results = []
    tpa.set_batch_width(0)
    default_width = tpa.get_batch_width()
    defaults = {}
    for w in widths:
        tpa.set_variant(w, -1)
        defaults[w] = tpa.get_variant(w)
    for w in widths:
        q = min(len(seeds), max(max_seeds if w >= 8 else 64, 2 * w))
        sd = torch.as_tensor(seeds[:q], dtype=torch.int32, device="cuda")
        out = torch.empty((n, q), dtype=torch.float32, device="cuda")
        tpa.set_batch_width(w)
        for v in tpa.variants():
            if v["kp"] != w:
                continue
            tpa.set_variant(w, v["index"])
            t = _time(lambda: tpa.query(g, sd, S, out=out), reps)
            results.append({"width": w, "variant": v["index"], "seeds_per_s": q / t})
        tpa.set_variant(w, -1)
    best = pick_query(results, defaults, default_width)
    tpa.set_batch_width(best["width"])
    tpa.set_variant(best["width"], best["variant"])
    return {"best": best, "all": results}


def autotune(g: tpa.Graph, seeds, c: float = 0.15, S: int = 5, T: int = 10, eps: float = 1e-9) -> dict:
    """Tune preprocessing and queries on graph g; leaves the best settings applied."""
    t0 = time.perf_counter()
    pre = tune_preprocess(g, c, T, eps)
    qry = tune_query(g, seeds, S)
    return {"preprocess": pre, "query": qry["best"], "candidates": len(qry["all"]) + 1,
            "seconds": time.perf_counter() - t0}
