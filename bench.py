"""Benchmark of the algebraic BFS on GB300.

Default workload: undirected R-MAT scale 22 (edge factor 16, a/b/c/d =
.57/.19/.19/.05, permuted labels), 16 sources drawn uniformly from the
vertices of degree >= 1.  One step = one BFS from each of the 16 sources
through the C-ABI (abfs_run), inputs resident in HBM.  The metric is GTEPS:
edges of the reached component (m_c = nnz_c / 2 for undirected graphs) over
device time.

Prints ONE JSON line (rank 0).  Under torchrun every rank runs the same
workload on its own GPU (independent replicas; BFS queries shard with no
exchange), value = all ranks' edges / max-over-ranks time.

--impl reference runs the CPU oracle (sorted-frontier queue BFS, one host
core) on the same workload, bounded to a few minutes.
--workload selects one of the other workloads (er16, grid4096, rgg22,
batch512, serve) for measurement runs; --workload ops prints the algebraic
operation counts of Section 11 (Table 2's columns) measured on the device for
the four single-graph workloads.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def _peaks():
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _engine_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1906_03113_gb300", "csrc")
    names = sorted(f for f in os.listdir(csrc) if f.startswith("engine") and f.endswith((".cu", ".cuh")))
    for f in names + ["internal.h"]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _profiled_traffic(workload: str):
    """(DRAM bytes per engine launch, ncu duration of that launch in us) from
    the committed ncu summary of this workload, or (None, None) when the
    engine source changed since the capture."""
    path = os.path.join(ROOT, "profiles", f"engine_kernel_{workload}.md")
    if not os.path.exists(path):
        return None, None
    fields = {}
    with open(path) as fh:
        for ln in fh:
            m = ln.strip().split(":", 1)
            if len(m) == 2 and m[0] in ("traffic_bytes_per_launch", "engine_source_sha256",
                                        "ncu_duration_us"):
                fields[m[0]] = m[1].strip()
    if fields.get("engine_source_sha256") != _engine_sha256():
        return None, None
    try:
        return int(fields["traffic_bytes_per_launch"]), float(fields.get("ncu_duration_us", "nan"))
    except (KeyError, ValueError):
        return None, None


def job_rate(units: float, ms: float, dist=None, device="cpu"):
    """Whole-job rate of independent replicas: the units (edges, queries) of
    all ranks over the slowest rank's time, per second; also that time in ms.
    No data moves between ranks except these two numbers."""
    if dist is not None:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        u = torch.tensor([units], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        ms, units = float(t.item()), float(u.item())
    return units / (ms * 1e-3), ms


def job_throughput(edges: float, ms: float, dist=None, device="cpu"):
    """job_rate for edges, in GTEPS."""
    rate, ms = job_rate(edges, ms, dist, device)
    return rate / 1e9, ms


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def make_workload(name: str):
    if name == "rmat22":
        g = synth.rmat_22()
        srcs = synth.sources_with_degree(g, 16, seed=1)
        desc = ("rmat22_16src", "R-MAT scale 22, edge factor 16, a/b/c/d=.57/.19/.19/.05, permuted, "
                "undirected, 16 sources from degree>=1 (seed 1)")
    elif name == "er16":
        g = synth.er_2_16()
        srcs = np.array([0], dtype=np.uint32)
        desc = ("er16_src0", "Erdos-Renyi G(n,p) n=2^16 p=8/(n-1) undirected, source 0 (seed 1)")
    elif name == "grid4096":
        g = synth.grid_4096()
        srcs = np.array([0], dtype=np.uint32)
        desc = ("grid4096_src0", "4096x4096 4-neighbour grid undirected, source 0")
    elif name == "rgg22":
        g = synth.rgg_2_22()
        srcs = np.array([0], dtype=np.uint32)
        desc = ("rgg22_src0", "directed 4-NN random geometric graph n=2^22, source 0 (seed 1)")
    else:
        raise ValueError(name)
    return g, srcs, desc


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    g, srcs, (wname, wdesc) = make_workload(args.workload)
    deg = g.degrees()
    directed = g.directed
    budget_s = 150.0
    # warm-up step (one source), also sizes the bounded sample
    t0 = time.perf_counter()
    lev, _ = oracle.bfs(g, int(srcs[0]))
    t_one = time.perf_counter() - t0
    steps = max(1, min(args.steps, int(budget_s / max(t_one, 1e-3))))
    edges, total = 0, 0.0
    for k in range(steps):
        s = int(srcs[k % len(srcs)])
        t0 = time.perf_counter()
        lev, _ = oracle.bfs(g, s)
        total += time.perf_counter() - t0
        nnz_c = int(deg[lev >= 0].sum())
        edges += nnz_c if directed else nnz_c // 2
    gteps = edges / total / 1e9
    line = {
        "impl": "reference", "metric": "GTEPS", "value": gteps, "unit": "GTEPS", "n_gpus": ws,
        "steps": steps, "steps_requested": args.steps, "warmup": 1,
        "ms_per_step": total / steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": wname, "graph": wdesc, "step": "one BFS from one source (rotating)"},
        "cpu_baseline": {"value": gteps, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                         "sample": f"{steps} single-source BFS of the workload, sources rotating"},
        "e2e": {"value": gteps, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def cpu_baseline(g, srcs, max_seconds=20.0):
    """The oracle (sorted-frontier queue BFS, one thread) on a bounded sample,
    and beside it the paper's own CPU methods: sequential Algorithm 2 and
    OpenMP Algorithm 3 on every host core (cpu_baselines/)."""
    import cpu_baselines
    import oracle
    deg = g.degrees()
    edges, total, used = 0, 0.0, 0
    for s in srcs:
        t0 = time.perf_counter()
        lev, _ = oracle.bfs(g, int(s))
        total += time.perf_counter() - t0
        used += 1
        nnz_c = int(deg[lev >= 0].sum())
        edges += nnz_c if g.directed else nnz_c // 2
        if total > max_seconds:
            break
    out = {"value": edges / total / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
           "sample": f"{used} of the {len(srcs)} sources, one BFS each, on one host core "
                     f"({total:.1f} s)",
           "host_cores": cpu_baselines.host_cores()}
    try:
        out["baselines"] = cpu_baselines.time_baselines(g, srcs, budget_s=max_seconds / 2, reps=5)
    except Exception as exc:  # a baseline that cannot run is reported, not fatal
        out["baselines"] = [{"error": f"{type(exc).__name__}: {exc}"}]
    return out


def _edges(st, directed):
    return st["nnz_reached"] if directed else st["nnz_reached"] / 2.0


def measure_batch(args, local, torch, abfs, big=None, G22=None, clocks=True):
    """512 ER/R-MAT graphs (n log-uniform in [2^10, 2^18], average degree U[4, 32])
    plus 64 sources on R-MAT-22, all in one persistent launch replayed from a
    CUDA graph, against the same queries as single-query launches.  Returns the
    measurements as a dict (big, G22: an R-MAT-22 graph already built)."""
    specs = synth.batch_specs(512, seed=1)
    hosts = [synth.make_batch_graph(sp) for sp in specs]
    own22 = big is None
    if own22:
        big = synth.rmat_22()
        G22 = abfs.graph_create(big.colptr, big.rowidx, directed=False)
    graphs = [abfs.graph_create(h.colptr, h.rowidx, directed=False) for h in hosts]
    srcs = [int(synth.sources_with_degree(h, 1, seed=1 + i)[0]) if (h.degrees() > 0).any() else 0
            for i, h in enumerate(hosts)]
    src22 = [int(x) for x in synth.sources_with_degree(big, 64, seed=2)]
    qg = graphs + [G22] * 64
    qs = srcs + src22
    qd = [h.directed for h in hosts] + [False] * 64
    stream = torch.cuda.current_stream()
    # edges of each query's component (from a counting run, outside the timing)
    edges = []
    lv = torch.empty(big.n, dtype=torch.int32, device="cuda")
    pv = torch.empty(big.n, dtype=torch.int32, device="cuda")
    for G, s_, d in zip(qg, qs, qd):
        _, _, st = abfs.run(G, s_, lv[:G.n], pv[:G.n], stream, None, stats=True)
        edges.append(_edges(st, d))
    total_edges = float(sum(edges))
    steps = max(1, min(args.steps, 20))
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)

    # parameters for the whole batch from the batch autotuner (outside the timing)
    tuned, tuned_ms = abfs.batch_tune(qg, qs)

    def batched_vs_single(gs, ss, clocks=None, params=None):
        params = tuned if params is None else params
        plan = abfs.BatchPlan(gs, ss, params=params)
        for _ in range(max(args.warmup, 3)):
            plan.launch(stream)
        torch.cuda.synchronize()
        assert all(x == 0 for x in plan.status()), "batch failed"
        if clocks is not None:
            clocks.start()
            time.sleep(0.3)
        a.record(stream)
        for _ in range(steps):
            plan.launch(stream)
        b.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks is not None else None
        bms = a.elapsed_time(b) / steps
        plan.destroy()
        # the same queries, one launch each
        a.record(stream)
        for G, s_ in zip(gs, ss):
            abfs.run(G, s_, lv[:G.n], pv[:G.n], stream, params)
        b.record(stream)
        torch.cuda.synchronize()
        return bms, a.elapsed_time(b), clk

    batch_ms, single_ms, clk = batched_vs_single(qg, qs, Clocks(local) if clocks else None)
    parts = {}
    for name, lo, hi in (("512_graphs", 0, len(graphs)), ("rmat22_64_sources", len(graphs), len(qg))):
        bms, sms, _ = batched_vs_single(qg[lo:hi], qs[lo:hi])
        e = float(sum(edges[lo:hi]))
        parts[name] = {"queries": hi - lo, "batched_ms": bms, "single_query_ms": sms,
                       "batched_gteps": e / (bms * 1e-3) / 1e9,
                       "single_query_gteps": e / (sms * 1e-3) / 1e9,
                       "speedup_vs_single": sms / bms}
    # the direction-optimising hybrid (not the paper's method) on the same queries
    hp = abfs.default_params(bottom_up_alpha=5, bottom_up_beta=24)
    hbms, hsms, _ = batched_vs_single(qg, qs, params=hp)
    hybrid = {"name": "direction-optimising hybrid, bottom_up_alpha 5, bottom_up_beta 24 "
                      "(not the paper's method)",
              "batched_ms": hbms, "batched_gteps": total_edges / (hbms * 1e-3) / 1e9,
              "single_query_ms": hsms, "speedup_vs_single": hsms / hbms}
    nq = len(qg)
    for G in graphs:
        G.destroy()
    if own22:
        G22.destroy()
    return {"queries": nq, "steps": steps, "warmup": max(args.warmup, 3), "ms": batch_ms,
            "total_edges": total_edges,
            "queries_per_s": nq / (batch_ms * 1e-3),
            "gteps": total_edges / (batch_ms * 1e-3) / 1e9,
            "single_query_ms": single_ms,
            "single_query_gteps": total_edges / (single_ms * 1e-3) / 1e9,
            "speedup_vs_single": single_ms / batch_ms, "parts": parts,
            "tuned_params": tuned.as_dict(), "tuner_ms": tuned_ms,
            "launch": "one persistent launch (CUDA graph replay) of all 576 queries, parameters "
                      "from the batch autotuner",
            "graph": "512 ER/R-MAT graphs, n log-uniform in [2^10, 2^18], avg degree U[4,32] "
                     "(seed 1), plus 64 sources on R-MAT-22 (seed 2)",
            "hybrid": hybrid, "clocks": clk}


def bench_batch(args, ws, rank, local, torch, abfs, dist):
    r = measure_batch(args, local, torch, abfs)
    value, _ = job_throughput(r["total_edges"], r["ms"], dist, "cuda")
    line = {
        "metric": "GTEPS", "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": r["steps"],
        "warmup": r["warmup"], "ms_per_step": r["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "batch512_rmat22x64", "graph": r["graph"],
                   "queries": r["queries"], "step": r["launch"],
                   "l2": "inputs larger than L2 (R-MAT-22 rowidx 513 MB, 576 workspaces)"},
        "batched": {k: r[k] for k in ("ms", "queries_per_s", "gteps", "single_query_ms",
                                      "single_query_gteps", "speedup_vs_single", "parts",
                                      "tuned_params", "tuner_ms")},
        "hybrid": r["hybrid"],
        "gpu_launches": 3 * r["steps"], "clocks": r["clocks"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_serve(args, torch, abfs):
    """32 resident graphs (16 R-MAT of scales 16..22, 15 ER of 2^16..2^20
    vertices, one 2048 x 2048 grid); queries with a uniform graph and source
    (degree >= 1) arrive as a Poisson stream at 0.5, 0.8 and 1.0 x the
    saturation rate measured first with a closed burst.  Returns a dict."""
    specs = synth.serve_graph_specs()
    hosts = [synth.make_serve_graph(k, kw) for k, kw in specs]
    graphs = [abfs.graph_create(h.colptr, h.rowidx, directed=False) for h in hosts]
    cand = [np.nonzero(h.degrees() > 0)[0].astype(np.int64) for h in hosts]
    rng = np.random.default_rng(1)
    nq = max(1000, args.queries)
    qg = rng.integers(len(hosts), size=nq)
    qs = np.array([cand[g][rng.integers(cand[g].size)] for g in qg], dtype=np.int64)
    pool = 48  # output buffers per graph
    bufs = [[(torch.empty(h.n, dtype=torch.int32, device="cuda"),
              torch.empty(h.n, dtype=torch.int32, device="cuda")) for _ in range(pool)]
            for h in hosts]
    cfg = abfs.serve_default_cfg(max_slots=256, memory_budget=48 << 30, idle_exit_ms=50)

    def run(rate, count):
        srv = abfs.Server(graphs, cfg)
        free = [list(range(pool)) for _ in hosts]
        outstanding = {}   # ticket -> (graph, buffer)
        waits = 0
        t0 = time.perf_counter()
        gap = np.random.default_rng(7).exponential(1.0 / rate, size=count) if rate else None
        t_next = t0
        for i in range(count):
            if rate:
                t_next += gap[i]
                while time.perf_counter() < t_next:
                    pass
            g = int(qg[i % nq])
            while not free[g]:
                waits += 1
                for t, (gg, bi) in list(outstanding.items()):
                    done, _ = srv.poll(t)
                    if done:
                        free[gg].append(bi)
                        del outstanding[t]
            bi = free[g].pop()
            lv, pv = bufs[g][bi]
            while True:
                t = srv.submit(g, int(qs[i % nq]), lv, pv)
                if t is not None:
                    break
            outstanding[t] = (g, bi)
            if len(outstanding) > 512 and i % 64 == 0:
                for t2, (gg, b2) in list(outstanding.items()):
                    done, _ = srv.poll(t2)
                    if done:
                        free[gg].append(b2)
                        del outstanding[t2]
        for t in list(outstanding):
            srv.wait(t, 600000)
        rep = srv.stop()
        rep["offered_qps"] = rate
        rep["buffer_waits"] = waits
        return rep

    # the same query stream as single-query launches (abfs_run, one per query, one stream)
    n_single = min(nq, 2000)
    stream = torch.cuda.current_stream()
    for i in range(8):
        g = int(qg[i])
        abfs.run(graphs[g], int(qs[i]), bufs[g][0][0], bufs[g][0][1], stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(n_single):
        g = int(qg[i])
        abfs.run(graphs[g], int(qs[i]), bufs[g][0][0], bufs[g][0][1], stream)
    torch.cuda.synchronize()
    single_qps = n_single / (time.perf_counter() - t0)

    sat = run(0.0, min(nq, 20000))              # closed burst: saturation throughput
    rates = [0.5, 0.8, 1.0]
    per = [run(f * sat["qps"], nq) for f in rates]
    for G in graphs:
        G.destroy()
    return {"queries_per_rate": nq, "sat": sat, "rates": rates, "per": per,
            "single_qps": single_qps, "n_single": n_single}


def serve_summary(r):
    """The serving figures of measure_serve's result."""
    best = r["per"][-1]
    return {
        "graph": "32 resident graphs: 16 R-MAT (scales 16..22), 15 ER (2^16..2^20, d=8), "
                 "one 2048x2048 grid",
        "queries_per_rate": r["queries_per_rate"],
        "arrivals": "Poisson at 0.5/0.8/1.0 x saturation",
        "saturation": {k: r["sat"][k] for k in ("qps", "p50_ms", "p99_ms", "completed", "launches")},
        "rates": [{k: x[k] for k in ("offered_qps", "qps", "p50_ms", "p99_ms", "mean_ms", "max_ms",
                                     "completed", "launches", "buffer_waits")} for x in r["per"]],
        "qps": best["qps"], "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"],
        "single_query": {"qps": r["single_qps"], "queries": r["n_single"],
                         "api": "abfs_run per query on one stream"},
        "speedup_vs_single": r["sat"]["qps"] / r["single_qps"],
    }


def bench_serve(args, ws, rank, local, torch, abfs, dist):
    r = measure_serve(args, torch, abfs)
    summ = serve_summary(r)
    best = r["per"][-1]
    job_qps, _ = job_rate(float(best["completed"]), best["wall_s"] * 1e3, dist, "cuda")
    line = {
        "metric": "queries/s", "value": job_qps, "unit": "queries/s", "n_gpus": ws,
        "steps": len(r["rates"]), "warmup": 1, "ms_per_step": best["wall_s"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "serve32_poisson", "graph": summ["graph"],
                   "queries_per_rate": summ["queries_per_rate"], "arrivals": summ["arrivals"]},
    }
    line.update({k: summ[k] for k in ("saturation", "rates", "p50_ms", "p99_ms", "single_query",
                                      "speedup_vs_single")})
    if rank == 0:
        print(json.dumps(line), flush=True)


def bench_ops(args, ws, rank, torch, abfs, dist):
    """Section 11's operation study (Table 2's columns) with the device counters.

    Per graph and source: Algorithm 2's 2(n_c - 1) (Theorem 2: one nonzero per
    reached row); the multiplies of Theorem 1's exact mask, 2 E_adj, every entry
    from level k into level k+1, counted by the submatrix engine as the entries
    that pass the mask; the all-nonzero variant of Algorithm 2 (Section 9), which
    Section 11 and Lemma 3 put at 2 m_c operations on an undirected graph
    (= nnz_c: each edge of the reached component is multiplied once, in the
    direction first scanned) -- order-dependent on directed graphs, so null
    there; masked SpMSpV's 2 nnz_c, counted by the comparator as the entries it
    multiplies; SpMV's 2 nnz L (closed form, not run).  Checks: the submatrix
    engine reads each reached column once (Claim 1, entries read = nnz_c),
    E_adj <= m, and the comparator multiplies exactly nnz_c entries."""
    rows = []
    t0 = time.perf_counter()
    for name in ("er16", "rmat22", "grid4096", "rgg22"):
        g, srcs, (wname, _) = make_workload(name)
        G = abfs.graph_create(g.colptr, g.rowidx, directed=g.directed)
        level = torch.empty(g.n, dtype=torch.int32, device="cuda")
        parent = torch.empty(g.n, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        m = g.nnz if g.directed else g.nnz // 2
        for s in srcs[:2]:
            _, _, sub = abfs.run(G, int(s), level, parent, stream, abfs.default_params(), stats=True)
            _, _, pl = abfs.run(G, int(s), level, parent, stream,
                                abfs.default_params(mode=abfs.MODE_PLAIN), stats=True)
            assert sub["status"] == 0 and pl["status"] == 0, (sub, pl)
            n_c, nnz_c, L = sub["reached"], sub["nnz_reached"], sub["levels"]
            e_adj = sub["entries_unmasked"]
            ops = {"alg2": 2 * (n_c - 1), "theorem1_multiplies": 2 * e_adj,
                   "alg2_all_nonzero": None if g.directed else nnz_c,
                   "spmmspv": 2 * pl["entries_read"], "spmv": 2 * g.nnz * L}
            checks = {"claim1_columns_once": sub["entries_read"] == nnz_c,
                      "lemma3_e_adj_le_m": e_adj <= m,
                      "spmmspv_eq_2nnz_c": pl["entries_read"] == nnz_c,
                      "same_levels": pl["levels"] == L and pl["reached"] == n_c}
            rows.append({"graph": wname, "source": int(s), "n": g.n, "m": m, "n_c": n_c,
                         "nnz_c": nnz_c, "levels": L, "e_adj": e_adj, "ops": ops,
                         "spmmspv_over_theorem1": ops["spmmspv"] / max(1, ops["theorem1_multiplies"]),
                         "spmmspv_over_all_nonzero": (None if g.directed else
                                                      ops["spmmspv"] / max(1, ops["alg2_all_nonzero"])),
                         "checks": checks})
        G.destroy()
    ok = all(all(r["checks"].values()) for r in rows)
    ratio = statistics.geometric_mean([r["spmmspv_over_theorem1"] for r in rows])
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps({
            "metric": "masked SpMSpV ops / Theorem 1 multiplies (geometric mean)",
            "value": ratio, "unit": "x", "n_gpus": ws, "steps": 1, "warmup": 0,
            "ms_per_step": (time.perf_counter() - t0) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "ops_table2", "graphs": "er16, rmat22 (2 sources), grid4096, rgg22",
                       "counts": "device counters of abfs_run with stats"},
            "all_checks_pass": ok, "rows": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat22",
                    choices=["rmat22", "er16", "grid4096", "rgg22", "batch512", "serve", "ops"])
    ap.add_argument("--queries", type=int, default=100000, help="serve: queries per arrival rate")
    ap.add_argument("--mode", default="sub", choices=["sub", "plain"])
    ap.add_argument("--shrink", type=float, default=0.0)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="library defaults instead of abfs_tune")
    ap.add_argument("--no-relabel", action="store_true",
                    help="rmat22: search the input numbering instead of abfs_graph_relabel's")
    ap.add_argument("--no-batch-serve", action="store_true",
                    help="default workload: skip the 576-query batch and the serving run")
    args = ap.parse_args()
    ws, rank, local = _dist()

    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    import paper_1906_03113_gb300 as abfs

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    abfs.load()
    if args.workload == "batch512":
        return bench_batch(args, ws, rank, local, torch, abfs, dist)
    if args.workload == "serve":
        return bench_serve(args, ws, rank, local, torch, abfs, dist)
    if args.workload == "ops":
        return bench_ops(args, ws, rank, torch, abfs, dist)

    g, srcs, (wname, wdesc) = make_workload(args.workload)
    G = abfs.graph_create(g.colptr, g.rowidx, directed=g.directed)
    # the skewed R-MAT graph runs on its copy renumbered by column-length class
    # (outputs still in the input's labels); the others keep their own order
    relabel = args.workload == "rmat22" and not args.no_relabel
    if relabel:
        abfs.graph_relabel(G)
    mode = abfs.MODE_PLAIN if args.mode == "plain" else abfs.MODE_SUBMATRIX
    # launch parameters for this graph from the library's autotuner (granule,
    # narrow bounds, cluster size, shrink threshold), on a few of the sources
    tune_srcs = srcs[:4]
    if args.no_tune:
        params, tune_ms = abfs.default_params(mode=mode), None
    else:
        params, tune_ms = abfs.tune(G, tune_srcs, mode)
    if args.shrink > 0:
        params.shrink_theta = args.shrink
        params.shrink_max = 1
    stream = torch.cuda.current_stream()
    n = g.n
    level = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")

    # per-source counters (outside the timed region)
    per_src = []
    for s in srcs:
        _, _, st = abfs.run(G, int(s), level, parent, stream, params, stats=True)
        assert st["status"] == 0, st
        per_src.append(st)
    nnz_c = np.array([st["nnz_reached"] for st in per_src], dtype=np.float64)
    m_c = nnz_c if g.directed else nnz_c / 2.0
    e_adj = np.array([st["entries_unmasked"] for st in per_src], dtype=np.float64)
    n_c = np.array([st["reached"] for st in per_src], dtype=np.float64)
    if mode == abfs.MODE_PLAIN:
        # the comparator multiplies every entry; E_adj comes from a submatrix run
        e_adj = []
        for s in srcs:
            _, _, st = abfs.run(G, int(s), level, parent, stream, abfs.default_params(), stats=True)
            e_adj.append(st["entries_unmasked"])
        e_adj = np.array(e_adj, dtype=np.float64)
    b_alg = 4.0 * e_adj + 24.0 * n_c           # algorithmic bytes per BFS
    b_cols = 4.0 * nnz_c + 24.0 * n_c          # bytes with every reached column read once

    def one_step():
        for s in srcs:
            abfs.run(G, int(s), level, parent, stream, params)

    for _ in range(max(args.warmup, 3)):
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()

    nsrc = len(srcs)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps * nsrc + 1)]
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    ev[0].record(stream)
    i = 0
    for _ in range(args.steps):
        for s in srcs:
            abfs.run(G, int(s), level, parent, stream, params)
            i += 1
            ev[i].record(stream)
    stop.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    edges_per_step = float(m_c.sum())
    value, total_ms = job_throughput(edges_per_step * args.steps, start.elapsed_time(stop), dist,
                                     "cuda")
    per_bfs_ms = np.array([ev[j].elapsed_time(ev[j + 1]) for j in range(args.steps * nsrc)])
    per_bfs_ms = per_bfs_ms.reshape(args.steps, nsrc).mean(axis=0)  # mean per source

    hbm, peak_kind = _peaks()
    mean_t = float(per_bfs_ms.mean()) * 1e-3
    achieved = float(b_alg.mean()) / mean_t / 1e9
    # the on-chip ceiling: every stored entry of a reached column costs one
    # random visited-bitmap load, every entry that passes the mask one random
    # reduction, both served by L2 (rates measured on this GPU, now)
    cal = abfs.calibrate(22)
    l2_bound_s = float(nnz_c.mean()) / (cal["load_gops"] * 1e9) + float(e_adj.mean()) / (
        cal["red_gops"] * 1e9)
    traffic, ncu_us = _profiled_traffic(wname)
    dram_gbs = traffic / (ncu_us * 1e-6) / 1e9 if traffic and ncu_us and ncu_us == ncu_us else None
    line = {
        "metric": "GTEPS", "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": wname, "graph": wdesc, "n": n, "nnz": g.nnz,
                   "sources": nsrc, "mode": args.mode, "shrink_theta": args.shrink,
                   "numbering": "abfs_graph_relabel: column-length classes (outputs in input "
                                "labels)" if relabel else "input",
                   "step": f"{nsrc} single-source BFS via abfs_run",
                   "l2": f"inputs larger than L2: rowidx {g.nnz * 4 / 1e6:.0f} MB",
                   "parallelism": f"replicas x{ws}", "edges": "m_c = nnz_c/2" if not g.directed
                   else "m_c = nnz_c",
                   "params": params.as_dict(),
                   "params_from": "defaults" if args.no_tune else
                   f"abfs_tune on {len(tune_srcs)} of the sources ({tune_ms:.3f} ms per search)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "peak_kind": peak_kind,
                     "traffic": traffic,
                     "dram_gbs": dram_gbs,
                     "dram_frac": None if dram_gbs is None else dram_gbs / hbm,
                     "dram_from": "ncu dram__bytes of one engine launch / its ncu duration "
                                  "(profiles/), null if the engine changed since",
                     "kernel": "engine_kernel<0> (one launch per BFS, after one initialisation "
                               "kernel" + (", before one relabel_out_kernel)" if relabel else ")"),
                     "bytes_per_bfs": float(b_alg.mean()),
                     "bytes_formula": "4*E_adj + 24*n_c",
                     "full_column_gbs": float(b_cols.mean()) / mean_t / 1e9,
                     "l2": {"random_load_gops": cal["load_gops"], "random_red_gops": cal["red_gops"],
                            "formula": "nnz_c / load rate + E_adj / red rate",
                            "bound_ms_per_bfs": l2_bound_s * 1e3,
                            "frac": l2_bound_s / mean_t}},
        "gpu_launches": (3 if relabel else 2) * nsrc * args.steps,
        "clocks": clk,
        "per_bfs_ms": float(per_bfs_ms.mean()),
        "reached_mean": float(n_c.mean()), "nnz_c_mean": float(nnz_c.mean()),
        "e_adj_mean": float(e_adj.mean()),
        "gteps_2m": value * (1.0 if g.directed else 2.0),
    }

    # end to end through host buffers: the step's searches in one abfs_run_host_many
    # call (each search's outputs leave for the host while the next one runs)
    lev_h = torch.empty((nsrc, n), dtype=torch.int32, pin_memory=True)
    par_h = torch.empty((nsrc, n), dtype=torch.int32, pin_memory=True)
    src_list = [int(s) for s in srcs]
    e2e_steps = max(1, min(args.steps, 10))
    abfs.run_host_many(G, src_list, lev_h, par_h, stream, params)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        _, _, st = abfs.run_host_many(G, src_list, lev_h, par_h, stream, params)
        assert all(x == 0 for x in st), st
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    # the same through one abfs_run_host call per search (no overlap), for context
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for s in src_list:
            abfs.run_host(G, s, lev_h[0], par_h[0], stream, params)
    torch.cuda.synchronize()
    single_s = time.perf_counter() - t0
    line["e2e"] = {"value": edges_per_step * e2e_steps * ws / e2e_s / 1e9, "unit": "GTEPS",
                   "h2d_bytes_per_step": 4 * nsrc, "d2h_bytes_per_step": 8 * n * nsrc,
                   "steps": e2e_steps,
                   "api": f"abfs_run_host_many: the step's {nsrc} searches in one call into "
                          "pinned host buffers",
                   "per_search_calls_gteps": edges_per_step * e2e_steps * ws / single_s / 1e9}

    if not args.no_extras and ws == 1:
        # comparator on the same GPU: plain masked SpMSpV (multiply, then mask),
        # tuned for itself in the same way
        pp = abfs.default_params(mode=abfs.MODE_PLAIN) if args.no_tune else \
            abfs.tune(G, tune_srcs, abfs.MODE_PLAIN)[0]
        for s in srcs:
            abfs.run(G, int(s), level, parent, stream, pp)
        torch.cuda.synchronize()
        c_steps = max(1, args.steps // 4)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(c_steps):
            for s in srcs:
                abfs.run(G, int(s), level, parent, stream, pp)
        b.record(stream)
        torch.cuda.synchronize()
        cms = a.elapsed_time(b)
        cval = edges_per_step * c_steps / (cms * 1e-3) / 1e9
        line["comparator"] = {"name": "plain masked SpMSpV (same engine, multiply then mask)",
                              "value": cval, "unit": "GTEPS", "speedup_of_ours": value / cval,
                              "params": pp.as_dict()}
        # same GPU, same search, two variants beside the paper's method: the
        # direction-optimising hybrid (bottom-up levels; identical results) and
        # the shortest-path counts of the all-nonzero variant (abfs_run_counts)
        def timed(fn, reps):
            for s in srcs[:2]:
                fn(int(s))
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(reps):
                for s in srcs:
                    fn(int(s))
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        hp = abfs.Params.from_buffer_copy(params)
        hp.bottom_up_alpha, hp.bottom_up_beta = 5, 24
        hp.shrink_theta, hp.shrink_max = 0.0, 0
        if not g.directed:
            hms = timed(lambda s: abfs.run(G, s, level, parent, stream, hp), c_steps)
            hval = edges_per_step / (hms * 1e-3) / 1e9
            line["hybrid"] = {"name": "direction-optimising hybrid (bottom-up levels over sorted "
                                      "columns, exact min-index parent; not the paper's method)",
                              "params": {"bottom_up_alpha": 5, "bottom_up_beta": 24},
                              "value": hval, "unit": "GTEPS", "per_bfs_ms": hms / nsrc,
                              "speedup_vs_submatrix": hval / value}
        sigma = torch.empty(n, dtype=torch.int64, device="cuda")
        cms2 = timed(lambda s: abfs.run_counts(G, s, level, parent, sigma, stream, params), c_steps)
        line["path_counts"] = {"name": "abfs_run_counts: shortest-path counts mod 2^64 (all-nonzero "
                                       "variant, arithmetic semiring)",
                               "value": edges_per_step / (cms2 * 1e-3) / 1e9, "unit": "GTEPS",
                               "per_bfs_ms": cms2 / nsrc,
                               "time_vs_abfs_run": cms2 / nsrc / float(per_bfs_ms.mean())}
        del sigma
        # batched: 64 sources in one persistent launch (CUDA graph replay)
        if args.workload == "rmat22":
            bs = synth.sources_with_degree(g, 64, seed=2)
            plan = abfs.BatchPlan([G] * 64, bs, params=params)
            plan.launch()
            torch.cuda.synchronize()
            assert all(x == 0 for x in plan.status())
            bm_c = []
            for s in bs:
                _, _, st = abfs.run(G, int(s), level, parent, stream, params, stats=True)
                bm_c.append(st["nnz_reached"] / 2.0)
            reps = 5
            a.record(stream)
            for _ in range(reps):
                plan.launch(stream)
            b.record(stream)
            torch.cuda.synchronize()
            bms = a.elapsed_time(b) / reps
            a.record(stream)
            for s in bs:
                abfs.run(G, int(s), level, parent, stream, params)
            b.record(stream)
            torch.cuda.synchronize()
            sms = a.elapsed_time(b)
            line["batched"] = {"queries": 64, "launch": "one persistent launch, CUDA graph replay",
                               "ms": bms, "gteps": sum(bm_c) / (bms * 1e-3) / 1e9,
                               "single_query_ms": sms,
                               "single_query_gteps": sum(bm_c) / (sms * 1e-3) / 1e9,
                               "speedup_vs_single": sms / bms}
            plan.destroy()

    if args.workload == "rmat22" and ws == 1 and not args.no_extras and not args.no_batch_serve:
        # the batch of 576 queries (512 graphs + 64 R-MAT-22 sources) and the
        # serving workload, measured in the same run
        try:
            line["batched_576"] = measure_batch(args, local, torch, abfs, big=g, G22=G, clocks=False)
            line["batched_576"].pop("clocks", None)
        except Exception as exc:
            line["batched_576"] = {"error": f"{type(exc).__name__}: {exc}"}
        try:
            line["serve"] = serve_summary(measure_serve(args, torch, abfs))
        except Exception as exc:
            line["serve"] = {"error": f"{type(exc).__name__}: {exc}"}

    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, srcs)
    G.destroy()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
