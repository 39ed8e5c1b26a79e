#!/usr/bin/env python
"""Benchmark of the TPA hot path on one GB300 (or N replicas).

Workload (one step): R-MAT scale 22 (4,194,304 nodes, 67,108,864 raw edges,
a/b/c/d = .57/.19/.19/.05, key 1; self-loops dropped and duplicates merged by
the graph builder), c = 0.15, S = 5, T = 10, eps = 1e-9:
  1. build the row-normalised CSR of A~^T and A~ from the edge list (resident in HBM),
  2. TPA preprocessing (Algorithm 2: PageRank CPI, stranger part from T on),
  3. 1,000 single-seed TPA queries (Algorithm 3), seeds uniform over nodes
     with an out-edge (key 2), answered in batches.
value = seeds answered per second over whole steps (all ranks).  Each rank is an
independent replica with its own 1,000 seeds (weak scaling, no data-path
collective).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (one query per step plus its 1/1000 share of the oracle's measured
build and preprocessing time).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "TPA seeds/s and SpMV HBM GB/s vs peak, batched vs per-seed CPI at L1≤1e-5"
C, S, T, EPS = 0.15, 5, 10, 1e-9
def workload(args) -> str:
    """The configuration a line measures, by what it is and its sizes."""
    return (f"TPA preprocessing + {args.queries} single-seed queries on R-MAT scale {args.scale} "
            f"(ef {args.edge_factor}), c={C} S={S} T={T} eps={EPS:.0e}".replace("e-0", "e-"))


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--edge-factor", type=int, default=16)
    ap.add_argument("--queries", type=int, default=1000)
    ap.add_argument("--batch", type=int, default=0, help="seeds per tpa_query call (0 = all at once)")
    ap.add_argument("--cpi-seeds", type=int, default=8, help="seeds for the per-seed exact CPI comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (library defaults)")
    ap.add_argument("--accuracy", type=int, default=0, metavar="SEEDS",
                    help="run the accuracy study of TPA's approximations (S sweep at T=10, T sweep at S=5, "
                         "recall@100/500) for SEEDS seeds on the GPU path, print one JSON line and exit")
    ap.add_argument("--graph", default="rmat", metavar="rmat|planted:BLOCKS:P_IN",
                    help="graph of the accuracy study: R-MAT (default) or a planted-partition graph with "
                         "BLOCKS equal communities and a share P_IN of edges inside them")
    ap.add_argument("--valued-products", action="store_true",
                    help="products that read the value array instead of the default pattern-only products")
    ap.add_argument("--serving", action="store_true",
                    help="measure batched serving instead: R-MAT --serving-scale (default 24), 8,192 seeds in "
                         "uneven batches of {1,7,32,100,256}, tpa_query per batch against CUDA-graph replays "
                         "(tpa_server); one JSON line")
    ap.add_argument("--serving-scale", type=int, default=24)
    ap.add_argument("--serving-seeds", type=int, default=8192)
    ap.add_argument("--adjoint", action="store_true",
                    help="measure the gradient of the link-prediction loss instead: R-MAT scale 20, 8 edge "
                         "features, 4,096 triples, K = the preprocessing count; one JSON line")
    ap.add_argument("--variant", action="append", default=[], metavar="NAME",
                    help="use the SpMV/SpMM variant NAME (e.g. 'seg<8,8,8>') for its padded width; repeatable")
    ap.add_argument("--profile-case", choices=["preprocess", "query8"], default=None,
                    help="run one small case for an ncu capture and exit (no JSON line): preprocessing of the "
                         "graph, or two 8-seed queries of light seeds after it")
    return ap.parse_args(argv)


def event_time(torch, fn, reps: int) -> float:
    """Seconds per call of fn (CUDA events on the current stream, after one warm-up call)."""
    fn()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / reps


def serving_study(args):
    """Batched serving (Algorithm 3 per request, batched): the seed stream in
    uneven batches answered by tpa_query per batch and by tpa_server replays;
    every timed pass follows an untimed one over the same batches."""
    import torch
    import synth
    import paper_1708_02574_gb300 as tpa
    tpa.set_pattern(not args.valued_products)
    apply_variants(tpa, args.variant)
    sc = args.serving_scale
    n = 1 << sc
    src, dst = synth.rmat_edges(sc, args.edge_factor)
    g = tpa.build_graph(n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    tpa.preprocess(g, C, T, EPS)
    cand = synth.nodes_with_out_edge(n, src, dst)
    total = args.serving_seeds
    seeds = synth.query_seeds(cand, total)
    sizes = synth.batch_sizes(total)
    m_raw = int(src.size)
    del src, dst
    batches, off = [], 0
    for k in sizes:
        batches.append(torch.from_numpy(seeds[off:off + k]).cuda())
        off += k
    srv = tpa.Server(g, S, max_k=max(sizes))
    clocks = ClockSampler(nvsmi_device_id())
    clocks.start()
    res = {}
    for name, run in (("direct", lambda b: tpa.query(g, b, S)), ("graphs", lambda b: srv.query(b))):
        def stream_pass():
            for b in batches:
                run(b)
        res[name] = total / event_time(torch, stream_pass, max(1, args.steps // 5))
    clk = clocks.stop()
    srv.sync()
    tpa.sync(g)
    st = srv.stats(256)
    line = {"study": "batched_serving", "metric": "seeds/s (uneven request batches, CUDA-graph replays)",
            "value": res["graphs"], "unit": "seeds/s", "higher_is_better": True, "data": "synthetic",
            "dtype": "f32", "direct_tpa_query_seeds_per_s": res["direct"],
            "graphs_over_direct": res["graphs"] / res["direct"],
            "config": {"workload": f"{total} seeds in uneven batches of {{1,7,32,100,256}} on R-MAT scale {sc} "
                                   f"(ef {args.edge_factor}), c={C} S={S} T={T}",
                       "n": n, "m": g.m, "m_raw": m_raw, "batches": len(sizes), "max_k": max(sizes)},
            "server": st, "clocks": clk}
    print(json.dumps(line), flush=True)
    srv.free()
    g.free()
    return 0


def adjoint_study(args):
    """Gradient of the link-prediction loss on TPA scores w.r.t. the edge-weight
    parameters: R-MAT scale 20, 8 features per edge ~ N(0,1), theta ~ N(0, 0.1^2),
    4,096 (seed, positive, negative) triples, K = the preprocessing count on the
    weighted graph.  One gradient = tpa_loss_grad + tpa_theta_grad."""
    import numpy as np
    import torch
    import synth
    import paper_1708_02574_gb300 as tpa
    apply_variants(tpa, args.variant)
    sc, ntrip, d = 20, 4096, 8
    n = 1 << sc
    src, dst = synth.rmat_edges(sc, 16)
    g = tpa.build_graph(n, src, dst)
    m = g.m
    feat = torch.from_numpy(synth.edge_features(m, d)).cuda()
    theta = torch.from_numpy(synth.theta(d)).cuda()
    cand = synth.nodes_with_out_edge(n, src, dst)
    seeds, pos, neg = synth.triples(n, src, dst, cand, ntrip)
    w = tpa.edge_weights(feat, theta)
    tpa.set_edge_weights(g, w)
    tpa.preprocess(g, C, T, EPS)
    K = max(int(tpa.get_stranger(g)[1]), T)
    sd, ps, ng = (torch.from_numpy(x).cuda() for x in (seeds, pos, neg))

    def grad():
        _, gw = tpa.loss_grad(g, sd, ps, ng, C, S, T, K)
        tpa.theta_grad(feat, w, gw)

    def loss_only():
        tpa.loss_grad(g, sd, ps, ng, C, S, T, K, want_grad=False)

    clocks = ClockSampler(nvsmi_device_id())
    clocks.start()
    t_grad = event_time(torch, grad, max(3, args.steps // 2))
    t_loss = event_time(torch, loss_only, max(3, args.steps // 2))
    clk = clocks.stop()
    # algorithmic bytes of one gradient: SpMVs over CSR(A~^T) and CSR(A~) at
    # 8m + 20n (k = 1) or 8m + 4n + 16nk (k = the family batch), edge passes at 16m (SDDMM:
    # row and column ids read, gradient read and written), the row Jacobian
    # at 16m, the theta reduction at (8 + 4d)m
    kb = tpa.get_adjoint_batch_width()   # triples per family batch
    batches = (ntrip + kb - 1) // kb
    spmv = s8d_bytes(n, m, 1)
    spmm = s8d_bytes(n, m, kb)
    alg = (K * spmv + batches * ((S - 1) * spmm + (S - 2) * spmm + (S - 1) * 16.0 * m)
           + K * spmv + K * 16.0 * m + 16.0 * m + (8.0 + 4.0 * d) * m)
    hbm, peak_kind = peaks()
    line = {"study": "adjoint", "metric": "gradients/s (loss + dL/dtheta over 4,096 triples)",
            "value": 1.0 / t_grad, "unit": "gradients/s", "higher_is_better": True, "data": "synthetic",
            "dtype": "f32 (fp64 reductions)", "ms_per_gradient": 1000.0 * t_grad,
            "ms_loss_only": 1000.0 * t_loss, "triples_per_s": ntrip / t_grad, "K": K, "family_batch": kb,
            "config": {"workload": f"link-prediction loss gradient, {ntrip} triples, R-MAT scale {sc} (ef 16), "
                                   f"{d} features, c={C} S={S} T={T}", "n": n, "m": m},
            "roofline": {"bound": "hbm", "achieved": alg / t_grad / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": alg / t_grad / 1e9 / hbm, "alg_bytes_per_gradient": alg,
                         "peak_source": f"{peak_kind} hbm_gbs (copy)"},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    g.free()
    return 0


def apply_variants(tpa, names):
    """Force the named kernel variants (tpa_set_variant) for their widths."""
    by_name = {v["name"]: v for v in tpa.variants()}
    for nm in names:
        v = by_name.get(nm)
        if v is None:
            raise SystemExit(f"unknown variant {nm!r}; known: {sorted(by_name)}")
        tpa.set_variant(v["kp"], v["index"])


def accuracy_study(args):
    """Errors of the neighbor and stranger approximations and of r_TPA against
    exact CPI (Table 3's quantities, the S and T sweeps of Section IV) on the
    R-MAT graph, SEEDS seeds uniform over nodes with an out-edge (key 2)."""
    import torch
    import synth
    import paper_1708_02574_gb300 as tpa
    from paper_1708_02574_gb300 import accuracy
    tpa.set_pattern(not args.valued_products)
    apply_variants(tpa, args.variant)
    n = 1 << args.scale
    if args.graph == "rmat":
        src, dst = synth.rmat_edges(args.scale, args.edge_factor)
        name = f"R-MAT scale {args.scale} ef {args.edge_factor}"
    else:
        kind, blocks, p_in = args.graph.split(":")
        assert kind == "planted", args.graph
        src, dst = synth.planted_edges(n, args.edge_factor, int(blocks), float(p_in))
        name = f"planted partition 2^{args.scale} nodes ef {args.edge_factor}, {blocks} blocks, p_in {p_in}"
    g = tpa.build_graph(n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    cand = synth.nodes_with_out_edge(n, src, dst)
    seeds = torch.from_numpy(synth.query_seeds(cand, args.accuracy)).cuda()
    t0 = time.perf_counter()
    res = accuracy.sweep(g, seeds, C, EPS, S_fixed=S, T_fixed=T, ks=(100, 500))
    print(json.dumps({"study": "tpa_accuracy", "data": "synthetic", "graph": name, "n": n, "m": g.m,
                      "c": C, "eps": EPS, "seeds": args.accuracy, "seconds": time.perf_counter() - t0, **res}))
    return 0


def profile_case(args):
    """A short, fixed sequence of library calls for kernel captures under ncu.

    preprocess: build the graph and run TPA preprocessing once (about 106 k = 1
    SpMV launches).  query8: the same, then two queries of 8 seeds with at most
    256 out-edges (push path for x1 and x2, then two pulled SpMM launches
    each, each with its fixup).  Library defaults, no tuning."""
    import torch
    import synth
    import paper_1708_02574_gb300 as tpa
    tpa.set_pattern(not args.valued_products)
    apply_variants(tpa, args.variant)
    n = 1 << args.scale
    src, dst = synth.rmat_edges(args.scale, args.edge_factor)
    g = tpa.build_graph(n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    tpa.preprocess(g, C, T, EPS)
    if args.profile_case == "query8":
        cand = synth.nodes_with_out_edge(n, src, dst)
        seeds = synth.query_seeds(cand, 64)
        rp, _, _ = tpa.get_csr(g, 1)
        deg = (rp[1:] - rp[:-1]).cpu().numpy()
        light = seeds[deg[seeds] <= 256][:8]
        sd = torch.from_numpy(light).cuda()
        for _ in range(2):
            tpa.query(g, sd, S)
    torch.cuda.synchronize()
    print(f"profile case {args.profile_case} done: n={n} m={g.m}", flush=True)
    return 0


# ------------------------------------------------------------ multi-rank ---
def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def shard_seeds(all_seeds, rank: int, world: int, per_rank: int):
    """Rank r answers seeds [r*per_rank, (r+1)*per_rank) of one global seed stream."""
    return all_seeds[rank * per_rank:(rank + 1) * per_rank]


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- clocks ---
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str):
        self.dev = device_id
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-i", self.dev, "-lms", "200"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            out = self.p.communicate(timeout=10)[0]
        except subprocess.TimeoutExpired:
            self.p.kill()
            out = self.p.communicate()[0]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def nvsmi_device_id() -> str:
    import torch
    try:
        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return "0"


# -------------------------------------------------------------- roofline ---
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    """Identity of the SpMV/SpMM device code (the files that define the kernels and Params)."""
    h = hashlib.sha256()
    for f in ("spmm_kernels.cuh", "spmm_binned.cuh", "spmm_lane.cuh"):
        with open(os.path.join(ROOT, "paper_1708_02574_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(variant: str, scale: int):
    """DRAM bytes (read + write) per launch of a kernel variant from a committed
    ncu capture, if it was taken on the current kernel source and graph scale.

    profiles/ncu_traffic.txt lines: variant source_hash scale bytes_per_launch note..."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    cur = kernel_source_hash()
    for line in open(path):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == variant and f[1] == cur and f[2] == str(scale):
            return float(f[3])
    return None


def bench_config(args, n: int, m: int, m_raw: int, world: int = 1) -> dict:
    """The workload a line measures; both arms print the same dict."""
    Q = args.queries
    return {"workload": workload(args), "graph": f"R-MAT scale {args.scale} ef {args.edge_factor}",
            "n": n, "m": m, "m_raw": m_raw, "queries_per_rank": Q, "query_batch": args.batch if args.batch > 0 else Q,
            "c": C, "S": S, "T": T, "eps": EPS, "parallelism": f"replicas x{world} (seed-sharded)",
            "products": "valued" if args.valued_products else "pattern-only",
            "l2": f"inputs larger than L2 (CSR {8 * m / 1e9:.1f} GB with values, scores {4 * n * Q / 1e9:.1f} GB "
                  f"per step)"}


def host_cpu() -> dict:
    """Core count and model of this host (the oracle's timing is quoted with it)."""
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu model", "hardware") and not model:
                model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if not model:   # Arm hosts name the core in lscpu only
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.split(":")[0].strip().lower() == "model name":
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count() or 1, "model": model}


def s8d_bytes(n: int, m: int, k: int) -> float:
    """Algorithmic bytes of one SpMV (k = 1) or k-column SpMM over CSR(A~^T):
    8m (column and value) + 20n for the SpMV, 8m + 4n + 16nk for the SpMM."""
    return 8.0 * m + 20.0 * n if k == 1 else 8.0 * m + 4.0 * n + 16.0 * n * k


# ------------------------------------------------------------ reference ---
def run_reference(args):
    """FP64 oracle on the host cores, bounded sample of the same workload."""
    import numpy as np
    import oracle
    import synth
    n = 1 << args.scale
    src, dst = synth.rmat_edges(args.scale, args.edge_factor)
    cand = synth.nodes_with_out_edge(n, src, dst)
    seeds = synth.query_seeds(cand, args.queries)
    t0 = time.perf_counter()
    og = oracle.build_graph(n, src, dst)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    rs, pre_it = oracle.preprocess(og, C, T, EPS)
    t_pre = time.perf_counter() - t0
    share = (t_build + t_pre) / args.queries
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.query(og, int(seeds[i % len(seeds)]), C, S, T, rs, EPS)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt + share)
    total = sum(times)
    value = len(times) / total
    host = host_cpu()
    sample = (f"oracle on {host['nproc']} OpenMP threads; per step: 1 oracle TPA query (4 SpMV over m={og.m}) "
              f"plus 1/{args.queries} of the oracle's measured CSR build ({t_build:.1f} s) and preprocessing "
              f"({t_pre:.1f} s, {pre_it} iterations)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "seeds/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": bench_config(args, n, og.m, int(src.size), args.gpus),
            "cpu_baseline": {"value": value, "unit": "seeds/s", "cores": host["nproc"], "kind": "oracle",
                             "sample": sample, "host": host},
            "e2e": {"value": value, "unit": "seeds/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- ours ---
def cpu_baseline(args, src, dst, seeds, gpu_pre_iters):
    """Time the oracle as it stands on a bounded sample, on one host core and on
    all of them (its loops over rows run on OpenMP threads; results are the
    same bits): the CSR build, 3 preprocessing iterations (scaled to the
    iteration count) and 2 queries (scaled to the query count).  `value` is
    the all-core estimate."""
    import numpy as np
    import oracle
    n = 1 << args.scale
    host = host_cpu()
    q = np.full(n, 1.0 / n)
    rs = np.zeros(n)
    est = {}
    try:
        for cores in (1, host["nproc"]):
            oracle.set_threads(cores)
            t0 = time.perf_counter()
            og = oracle.build_graph(n, src, dst)
            t_build = time.perf_counter() - t0
            t0 = time.perf_counter()
            oracle.cpi(og, q, C, EPS, T, 3)
            t_it = (time.perf_counter() - t0) / 3
            t0 = time.perf_counter()
            for sd in seeds[:2]:
                oracle.query(og, int(sd), C, S, T, rs, EPS)
            t_q = (time.perf_counter() - t0) / 2
            total = t_build + gpu_pre_iters * t_it + args.queries * t_q
            est[cores] = (args.queries / total, t_build, t_it, t_q)
            del og
    finally:
        oracle.set_threads(0)
    one, allc = est[1], est[host["nproc"]]
    return {"value": allc[0], "unit": "seeds/s", "cores": host["nproc"], "kind": "oracle", "host": host,
            "single_core": {"value": one[0], "cores": 1},
            "sample": (f"oracle on {host['nproc']} threads: CSR build timed in full ({allc[1]:.1f} s), 3 "
                       f"preprocessing iterations ({allc[2]:.3f} s each) scaled to {gpu_pre_iters}, 2 queries "
                       f"({allc[3]:.3f} s each) scaled to {args.queries}; on 1 thread {one[1]:.1f} s, "
                       f"{one[2]:.3f} s and {one[3]:.3f} s")}


def main(argv=None):
    args = parse_args(argv)
    if args.profile_case:
        return profile_case(args)
    if args.accuracy:
        return accuracy_study(args)
    if args.serving:
        return serving_study(args)
    if args.adjoint:
        return adjoint_study(args)
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return 0

    import numpy as np
    import torch
    import synth
    import paper_1708_02574_gb300 as tpa

    tpa.set_pattern(not args.valued_products)
    apply_variants(tpa, args.variant)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = 1 << args.scale
    src, dst = synth.rmat_edges(args.scale, args.edge_factor)
    cand = synth.nodes_with_out_edge(n, src, dst)
    all_seeds = synth.query_seeds(cand, args.queries * world)
    seeds = shard_seeds(all_seeds, rank, world, args.queries)
    Q = len(seeds)
    src_d = torch.from_numpy(src).cuda()
    dst_d = torch.from_numpy(dst).cuda()
    seeds_d = torch.from_numpy(seeds).cuda()
    out_d = torch.empty((n, Q), dtype=torch.float32, device="cuda")
    batch = args.batch if args.batch > 0 else Q

    # untimed setup: tune kernel variants and the batch width on this graph and seed mix
    from paper_1708_02574_gb300 import autotune
    g0 = tpa.build_graph(n, src_d, dst_d)
    tpa.preprocess(g0, C, T, EPS)
    tuned = autotune.autotune(g0, seeds, C, S, T, EPS) if not args.no_tune else None
    g0.free()

    def step():
        g = tpa.build_graph(n, src_d, dst_d)
        tpa.preprocess(g, C, T, EPS)
        if batch >= Q:
            tpa.query(g, seeds_d, S, out=out_d)
        else:
            for j0 in range(0, Q, batch):
                tpa.query(g, seeds_d[j0:j0 + batch], S, out=torch.empty((n, min(batch, Q - j0)),
                                                                          dtype=torch.float32, device="cuda"))
        g.free()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    clocks = ClockSampler(nvsmi_device_id()) if rank == 0 else None
    if clocks:
        clocks.start()
    tpa.profile_reset(timing=True)
    l0 = tpa.launch_count()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nvtx = getattr(torch.cuda, "nvtx", None)
    try:
        nvtx.range_push("bench_timed")    # lets a profiler select the timed steps only
    except Exception:
        nvtx = None
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    if nvtx is not None:
        nvtx.range_pop()
    torch.cuda.synchronize()
    barrier(world)
    launches = tpa.launch_count() - l0
    stats = tpa.profile_read()
    tpa.profile_reset(timing=False)
    clk = clocks.stop() if clocks else None
    t_rank = e0.elapsed_time(e1) / 1000.0
    t = max_over_ranks(t_rank, world)
    value = Q * world * args.steps / t

    # phase breakdown and per-seed exact CPI on the same GPU (untimed by the contract)
    g = tpa.build_graph(n, src_d, dst_d)
    m = g.m
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    g.free()
    g = tpa.build_graph(n, src_d, dst_d)
    ev[1].record(stream)
    tpa.preprocess(g, C, T, EPS)
    ev[2].record(stream)
    tpa.query(g, seeds_d, S, out=out_d)
    ev[3].record(stream)
    torch.cuda.synchronize()
    _, pre_iters = tpa.get_stranger(g)
    phases = {"build": ev[0].elapsed_time(ev[1]), "preprocess": ev[1].elapsed_time(ev[2]),
              "queries": ev[2].elapsed_time(ev[3])}
    cpi_seeds = seeds[:args.cpi_seeds]
    tpa.cpi_exact(g, int(cpi_seeds[0]), C, EPS)
    torch.cuda.synchronize()
    c0 = time.perf_counter()
    for sd in cpi_seeds:
        tpa.cpi_exact(g, int(sd), C, EPS)
    torch.cuda.synchronize()
    cpi_sps = len(cpi_seeds) / (time.perf_counter() - c0)
    # like-for-like: exact CPI for a batch of seeds through the batched path
    bseeds = seeds_d[:64]
    tpa.cpi(g, bseeds, C, EPS)
    torch.cuda.synchronize()
    c0 = time.perf_counter()
    tpa.cpi(g, bseeds, C, EPS)
    torch.cuda.synchronize()
    bcpi_sps = len(bseeds) / (time.perf_counter() - c0)

    # batched serving: uneven request batches (sizes uniform over {1,7,32,100,256})
    # through tpa_query per batch and through a tpa_server replaying CUDA graphs
    try:
        serving = measure_serving(tpa, torch, g, cand, stream)
    except tpa.TpaError as e:   # e.g. the server's n x 256 output does not fit beside the graph
        serving = {"unavailable": str(e)[:200]}

    hbm, peak_kind = peaks()

    # the gathers alone at this column pattern (tpa_probe_gather), the floor
    # the SpMV/SpMM launches are compared with in the roofline objects
    probe_ms = {kp: tpa.probe_gather(g, kp, reps=5) for kp in (1, 8)}

    names = {v["index"]: v["name"] for v in tpa.variants()}

    def roofline_of(fam):
        sp = stats.get(fam, {})
        if sp.get("total_ms", 0) <= 0:
            return None
        kp = int(fam[len("spmm_kp"):])
        # one SpMV/SpMM = the walk and, for the lane-segment walk, its finishing
        # launch (rows, epilogue, L1 norm, break test), timed as finish_kpK
        fin = stats.get(f"finish_kp{kp}", {})
        walk_s = sp["total_ms"] / 1000.0 / max(1, sp["launches"])
        fin_s = fin.get("total_ms", 0.0) / 1000.0 / max(1, fin.get("launches", 0)) if fin.get("launches") else 0.0
        avg_s = walk_s + fin_s
        # the contract's bytes: 8m + 20n per SpMV, 8m + 4n + 16nk per k-column
        # SpMM (every launch of the bench's chunks has k = kp columns)
        per_launch = s8d_bytes(n, m, kp)
        achieved = per_launch / avg_s / 1e9
        moved = sp["alg_bytes"] / max(1, sp["launches"])   # what the kernel reads and writes itself
        variant = names.get(tpa.get_variant(kp), "?")
        products = "valued" if args.valued_products else "pattern"
        traffic = ncu_traffic(f"{variant}+{products}", args.scale)
        return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "variant": variant,
                # DRAM GB/s from the ncu bytes over this run's launch time, and
                # its ratio to the algorithmic bytes (gather over-fetch when > 1)
                "dram_gbs": traffic / avg_s / 1e9 if traffic else None,
                "traffic_over_alg": traffic / per_launch if traffic else None,
                # edges traversed per second (each nonzero of CSR(A~^T) once per launch)
                "gteps": m / avg_s / 1e9,
                # one pass of the gathers alone (column ids in order, a row of kp
                # floats gathered per nonzero, no row logic) and the launch over it
                "gather_probe_ms": probe_ms.get(kp),
                "launch_over_gather_probe": 1000.0 * avg_s / probe_ms[kp] if probe_ms.get(kp) else None,
                "products": products,
                "kernel": (f"{fam} + finish_kp{kp}" if fin_s else fam)
                          + f": SpMV/SpMM over CSR(A~^T), {variant}, {products} products",
                "launches": sp["launches"], "avg_launch_ms": 1000.0 * avg_s,
                "walk_ms": 1000.0 * walk_s, "finish_ms": 1000.0 * fin_s,
                "alg_bytes_per_launch": per_launch,
                "alg_bytes_rule": "8m + 20n (k = 1) or 8m + 4n + 16nk per launch, m after merging duplicates",
                "moved_bytes_per_launch": moved, "achieved_moved": moved / avg_s / 1e9,
                "frac_moved": moved / avg_s / 1e9 / hbm,
                "peak_source": f"{peak_kind} hbm_gbs (copy), burst",
                "kernel_share_of_step": (sp["total_ms"] + fin.get("total_ms", 0.0)) / (1000.0 * t_rank)}

    fams = [f for f in stats if f.startswith("spmm_kp")]
    dominant = max(fams, key=lambda f: stats[f]["total_ms"]) if fams else None
    roof = roofline_of(dominant) if dominant else None
    roof_k1 = roofline_of("spmm_kp1")

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(args, tpa, torch, n, src, dst, seeds)

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(args, src, dst, seeds, pre_iters)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "seeds/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000.0 * t / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": bench_config(args, n, m, int(src.size), world),
                "roofline": roof, "cpu_baseline": base, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk,
                "phases_ms": phases, "preprocess_iters": pre_iters,
                "online_seeds_per_s": Q / (phases["queries"] / 1000.0),
                "per_seed_cpi": {"value": cpi_sps, "unit": "seeds/s", "seeds": len(cpi_seeds), "eps": EPS},
                "batched_cpi": {"value": bcpi_sps, "unit": "seeds/s", "seeds": int(bseeds.numel()), "eps": EPS},
                "roofline_spmv_k1": roof_k1, "serving": serving, "autotune": tuned, "kernels": stats}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def measure_serving(tpa, torch, g, cand, stream, total=2048):
    """Seeds/s of a stream of uneven batches, direct tpa_query calls against
    CUDA-graph replays (tpa_server), each after one untimed pass over the sizes."""
    import synth
    sizes = synth.batch_sizes(total)
    seeds = synth.query_seeds(cand, total, key=5)
    batches, off = [], 0
    for k in sizes:
        batches.append(torch.from_numpy(seeds[off:off + k]).cuda())
        off += k
    out = torch.empty((g.n, max(sizes)), dtype=torch.float32, device="cuda")
    try:
        srv = tpa.Server(g, S, max_k=max(sizes), out=out)
    except tpa.TpaError as e:       # the server refuses graphs above its validated size
        return {"unavailable": str(e)}
    res = {"batches": len(sizes), "seeds": total, "sizes": sorted(set(sizes))}
    try:
        for name, run in (("direct", lambda b: tpa.query(g, b, S)),
                          ("graphs", lambda b: srv.query(b))):
            for b in batches:
                run(b)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for b in batches:
                run(b)
            e1.record(stream)
            torch.cuda.synchronize()
            res[name + "_seeds_per_s"] = total / (e0.elapsed_time(e1) / 1000.0)
        res["server"] = srv.stats(max(sizes))
    finally:
        srv.free()
        del out
    return res


def measure_e2e(args, tpa, torch, n, src, dst, seeds):
    """Same step through the C ABI with host buffers: edges from pinned host memory,
    scores read back into pinned host memory, copies inside the timed region."""
    Q = len(seeds)
    src_h = torch.from_numpy(src).pin_memory()
    dst_h = torch.from_numpy(dst).pin_memory()
    seeds_h = torch.from_numpy(seeds).pin_memory()
    out_h = torch.empty((n, Q), dtype=torch.float32, pin_memory=True)

    def step():
        g = tpa.build_graph(n, src_h, dst_h)
        tpa.preprocess(g, C, T, EPS)
        tpa.query(g, seeds_h, S, out=out_h)
        g.free()

    step()
    torch.cuda.synchronize()
    k = max(3, args.steps)
    t0 = time.perf_counter()
    for _ in range(k):
        step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    # what the host link gives a plain copy of the same bytes (tpa_query
    # copies the scores by column groups while the next group computes)
    link = {}
    try:
        dev = torch.empty((n, Q), dtype=torch.float32, device="cuda")
        dev.fill_(1.0)
        srcd = torch.empty(src.size, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        for name, dst_t, src_t in (("d2h", out_h, dev), ("h2d", srcd, src_h)):
            dst_t.copy_(src_t, non_blocking=True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                dst_t.copy_(src_t, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            nbytes = src_t.numel() * src_t.element_size()
            link[f"{name}_copy_gbs"] = 3 * nbytes / (e0.elapsed_time(e1) / 1000.0) / 1e9
            link[f"{name}_copy_bytes"] = int(nbytes)
        del dev, srcd
    except RuntimeError as e:   # not enough device memory for the copy test
        link = {"unavailable": str(e)[:200]}
    del out_h
    return {"value": Q * k / dt, "unit": "seeds/s", "steps": k, "ms_per_step": 1000.0 * dt / k,
            "h2d_bytes_per_step": int(src.nbytes + dst.nbytes + seeds.nbytes),
            "d2h_bytes_per_step": int(4 * n * Q), "host_link_plain_copy": link}


if __name__ == "__main__":
    sys.exit(main())
