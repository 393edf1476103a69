#!/usr/bin/env python
"""Benchmark of the constraint-checking pruning pipeline on one GB300.

One step = one pass of the whole hot path (init, LCC to fixpoint, every
non-local constraint with LCC re-runs, final template-driven search with
match counting) for each template of the workload, over a resident synthetic
R-MAT graph.  Default workload: R-MAT scale 22, edge factor 16, degree labels,
two 6-vertex templates (an acyclic tree that LCC alone settles, and a template
with a 4-cycle and a triangle that needs non-local constraints).

value  = edges scanned per second (active CSR entries read by LCC rounds plus
         CSR entries examined by searches), device time, inputs resident.
e2e    = the same metric through the C ABI with pinned host buffers: graph
         upload, pruning, read-back of omega and the edge bitmap to the host.
Under torchrun each rank runs its own replica (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "template time-to-solution (ms) & edges scanned/s, batched+learned vs plain"
# "edges scanned" counts the active CSR entries the LCC rounds examine: the
# same number on every implementation that follows the method (the GPU path
# and the oracle agree on it bit for bit), so values of different arms compare
# as time ratios.  Entries examined by the searches depend on how a search is
# organised and are reported beside it, not in it.

WORKLOADS = {
    "rmat22-degree": {
        "scale": 22, "labels": "degree",
        "templates": {
            "tree6": ([11, 3, 6, 8, 7, 9], [(0, 1), (1, 2), (1, 3), (3, 4), (4, 5)]),
            "c4tri6": ([5, 12, 11, 11, 5, 7], [(0, 1), (1, 2), (2, 3), (3, 0), (2, 4), (3, 4), (4, 5)]),
        },
    },
    # many templates over one resident graph: 64 edit-distance variants (k = 1, 2)
    # of the 4-cycle + triangle template, pruned one at a time in the fixed
    # order (plain) and batched with the learned order
    "batch22": {
        "scale": 22, "labels": "degree", "batch": 64, "batch_seed": 5,
        "templates": {
            "c4tri6": ([5, 12, 11, 11, 5, 7], [(0, 1), (1, 2), (2, 3), (3, 0), (2, 4), (3, 4), (4, 5)]),
        },
    },
    "rmat16-degree": {
        "scale": 16, "labels": "degree",
        "templates": {
            "treetri6": ([5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)]),
        },
    },
}

SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ccpm", "reference"], default="ccpm")
    p.add_argument("--workload", default="rmat22-degree", choices=sorted(WORKLOADS))
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--count-cap", type=int, default=1 << 30,
                   help="matches counted per template before the count is reported invalid "
                        "(omega* and E* stay exact)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def make_graph(wl_cfg, device=None):
    from paper_1912_08453_gb300 import workloads as wl
    return wl.rmat_graph(wl_cfg["scale"], labels=wl_cfg["labels"], device=device)


class ClockSampler:
    """nvidia-smi sampling during the timed region (every 200 ms)."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ccpm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={SMI_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9], parts[4]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


def kernel_source_hash():
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_1912_08453_gb300", "csrc", "ccpm_kernels.cu"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """Average DRAM bytes per launch of `kernel` over the timed step, from the
    committed ncu summary, only if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", f"dram_{workload}.md")
    if not os.path.exists(path):
        return None
    src, traffic = None, None
    for line in open(path):
        if line.startswith("kernel-source-sha256:"):
            src = line.split(":", 1)[1].strip()
        if line.startswith(f"dram-bytes-per-launch {kernel}:"):
            traffic = float(line.split(":", 1)[1].strip())
    if src != kernel_source_hash():
        return None
    return traffic


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def cpu_oracle_run(g, templates, budget_s=30.0):
    """The CPU oracle as it stands, single-threaded, on the same graph: whole
    templates until about budget_s seconds of CPU work have been spent."""
    from oracle import pipeline
    done, edges, secs = [], 0, 0.0
    for name, (tl, te) in templates.items():
        r = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
        edges += r.lcc_scanned
        secs += r.seconds
        done.append(f"{name}: {r.seconds:.1f}s")
        if secs > budget_s:
            break
    return edges, secs, done


def run_reference(args, cfg):
    """Reference arm: the CPU oracle timed on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    g = make_graph(cfg)
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; nothing to do
    times, edges = [], 0
    sample = dict(cfg["templates"])          # the same templates as the GPU arm's step
    for _ in range(args.steps):
        e, s, _ = cpu_oracle_run(g, sample, budget_s=1e9)
        edges += e
        times.append(s)
    total = sum(times)
    value = edges / total if total > 0 else 0.0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges scanned/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": args.workload, "scale": cfg["scale"], "n": g.n, "m_dir": g.m_dir,
                       "templates": sorted(sample)},
            "cpu_baseline": {"value": value, "unit": "edges scanned/s", "cores": 1, "kind": "oracle",
                             "sample": "every template of the workload per step, whole pipeline"},
            "e2e": {"value": value, "unit": "edges scanned/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def graph_workers(graph):
    """Worker count the batch autotuner chose for this graph."""
    from paper_1912_08453_gb300 import ccpm
    return int(ccpm.lib.ccpm_graph_batch_workers(graph.h))


def batch_templates(cfg):
    from paper_1912_08453_gb300 import workloads as wl
    (name, (tl, te)), = cfg["templates"].items()
    base = wl.Template(list(tl), list(te), name=name)
    pool = sorted(set(tl))
    return [base] + wl.edit_variants(base, cfg["batch"] - 1, seed=cfg["batch_seed"], label_pool=pool)


def run_batch_workload(args, cfg):
    """Plain (one template at a time, fixed order) vs batched + learned order.
    Under torchrun the templates are dealt to the ranks (longest first, by
    rank 0's warm-up times); each rank prunes its share over its own copy of
    the graph, and the step time is the maximum over ranks."""
    import torch
    from paper_1912_08453_gb300.build import build
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1912_08453_gb300 import ccpm, ordering, sharding
    g = make_graph(cfg, device=f"cuda:{local}")
    torch.cuda.empty_cache()
    stream = torch.cuda.Stream()
    ctx = ccpm.Context(local, stream=stream.cuda_stream)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    tmpls_all = batch_templates(cfg)
    hs_all = [ccpm.Template(ctx, t.labels, t.edges) for t in tmpls_all]
    cap = ccpm.options(max_embeddings=args.count_cap)

    def plain(results):
        for i, h in enumerate(hs):
            results[i] = ccpm.prune(ctx, graph, h, cap, result=results[i], allow_budget=True)
        return results

    def timed(fn):
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        out = fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return out, ev0.elapsed_time(ev1)

    with torch.cuda.stream(stream):
        # warm-up over every template; rank 0's times deal the templates
        res_all = [None] * len(hs_all)
        for _ in range(args.warmup):
            for i, h in enumerate(hs_all):
                res_all[i] = ccpm.prune(ctx, graph, h, cap, result=res_all[i], allow_budget=True)
        costs = torch.tensor([r.counts()["ms_total"] for r in res_all], dtype=torch.float64,
                             device=f"cuda:{local}")
        if world > 1:
            torch.distributed.broadcast(costs, 0)
        mine = sharding.deal(costs.tolist(), world)[rank]
        hs = [hs_all[i] for i in mine]
        tmpls = [tmpls_all[i] for i in mine]
        res_plain = [res_all[i] for i in mine]
        # the plain pipeline's own logs train the ordering network
        recs = [rec for r in res_plain for rec in r.logs()]
        X, y = ordering.targets_from(recs)
        net = ordering.train(ctx, X, y, steps=2000) if len(recs) >= 8 else None
        learned = ordering.learned_options(net, max_embeddings=args.count_cap) if net else cap
        res_batch = ccpm.prune_batch(ctx, graph, hs, learned, allow_budget=True)   # autotunes workers
        res_bfix = ccpm.prune_batch(ctx, graph, hs, cap, allow_budget=True)
        res_plearn = [None] * len(hs)
        t_plain, t_batch, t_bfix, t_plearn = [], [], [], []
        for _ in range(args.steps):
            _, ms = timed(lambda: plain(res_plain))
            t_plain.append(ms)
            _, ms = timed(lambda: ccpm.prune_batch(ctx, graph, hs, learned, results=res_batch, allow_budget=True))
            t_batch.append(ms)
            _, ms = timed(lambda: ccpm.prune_batch(ctx, graph, hs, cap, results=res_bfix, allow_budget=True))
            t_bfix.append(ms)

            def plain_learned():
                for i, h in enumerate(hs):
                    res_plearn[i] = ccpm.prune(ctx, graph, h, learned, result=res_plearn[i], allow_budget=True)
            _, ms = timed(plain_learned)
            t_plearn.append(ms)
    same = all(np.array_equal(a.omega(), b.omega()) and np.array_equal(a.edge_bitmap(), b.edge_bitmap())
               and a.counts()["match_embeddings"] == b.counts()["match_embeddings"]
               for a, b in zip(res_plain, res_batch))
    edges = sum(r.counts()["edges_scanned_lcc"] for r in res_batch)
    ms_plain, ms_batch = statistics.median(t_plain), statistics.median(t_batch)
    dev = f"cuda:{local}"
    ms_plain, _, _ = sharding.reduce_step(ms_plain, 0, True, device=dev)
    ms_batch, edges, same = sharding.reduce_step(ms_batch, edges, same, device=dev)
    ms_bfix, _, _ = sharding.reduce_step(statistics.median(t_bfix), 0, True, device=dev)
    ms_plearn, _, _ = sharding.reduce_step(statistics.median(t_plearn), 0, True, device=dev)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": edges / (ms_batch / 1e3), "unit": "edges scanned/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": args.workload, "graph": f"R-MAT scale {cfg['scale']}, degree labels",
                       "n": g.n, "m_dir": g.m_dir, "templates": len(hs_all), "templates_rank0": len(hs),
                       "template_sizes": sorted({t.n0 for t in tmpls_all}),
                       "parallelism": f"templates dealt over {world} ranks" if world > 1 else "one GPU",
                       "l2": "inputs larger than L2 (the 513 MB column array)"},
            "plain_ms": ms_plain, "batched_learned_ms": ms_batch, "speedup": ms_plain / ms_batch,
            "batched_fixed_ms": ms_bfix, "plain_learned_ms": ms_plearn,
            "plain_split_ms": {k: sum(r.counts()[k] for r in res_plain) for k in ("ms_lcc", "ms_nlcc", "ms_final")},
            "count_cap": args.count_cap,
            "counts_valid": int(sum(r.counts()["count_valid"] for r in res_plain)),
            "workers": graph_workers(graph),
            "identical_outputs": bool(same),
            "matches_total": int(sum(r.counts()["match_embeddings"] for r in res_batch)),
            "training_records": len(recs)}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    cfg = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, cfg)
        return
    if "batch" in cfg:
        run_batch_workload(args, cfg)
        return
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1912_08453_gb300.build import build
    if rank == 0 or world == 1:
        build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1912_08453_gb300 import ccpm

    g = make_graph(cfg, device=f"cuda:{local}")
    torch.cuda.empty_cache()
    stream = torch.cuda.Stream()
    ctx = ccpm.Context(local, stream=stream.cuda_stream)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    tmpls = {k: ccpm.Template(ctx, tl, te) for k, (tl, te) in cfg["templates"].items()}
    results = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")

    def one_step():
        stats = {}
        for k, t in tmpls.items():
            r = ccpm.prune(ctx, graph, t, result=results.get(k))
            results[k] = r
            stats[k] = r.counts()
        return stats

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            one_step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        step_ms, agg = [], []
        for _ in range(args.steps):
            flush.zero_()                      # L2 flush between timed steps
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            st = one_step()
            ev1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            agg.append(st)
        clk = clocks.stop()
    edges = sum(c["edges_scanned_lcc"] for st in agg for c in st.values())
    search_entries = sum(c["edges_scanned_search"] for st in agg for c in st.values())
    total_ms = sum(step_ms)
    from paper_1912_08453_gb300 import sharding
    total_ms, edges, _ = sharding.reduce_step(total_ms, edges, True, device=f"cuda:{local}")
    value = edges / (total_ms / 1e3)
    tts = {k: statistics.mean(st[k]["ms_total"] for st in agg) for k in tmpls}

    # rooflines of the two kernels that take the time: the LCC round (algorithmic
    # bytes: 24 per active vertex, 4.125 per row entry, 4 per active entry) and
    # the NLCC search (8 per row entry examined: the column index and the
    # neighbour's omega); "roofline" is the one with more device time
    peak, peak_kind = measured_peak_hbm()

    def roof(kernel, alg_bytes, ms, n_launch):
        achieved = (alg_bytes / 1e9) / (ms / 1e3) if ms > 0 else 0.0
        return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": recorded_traffic(kernel, args.workload),
                "alg_bytes_per_launch": alg_bytes / max(n_launch, 1),
                "avg_launch_ms": ms / max(n_launch, 1), "launches": n_launch, "device_ms": ms}

    every = [c for st in agg for c in st.values()]
    roof_lcc = roof("k_lcc_round", sum(c["lcc_alg_bytes"] for c in every), sum(c["ms_lcc_kernel"] for c in every),
                    sum(c["lcc_launches"] for c in every))
    roof_search = roof("k_nlcc_items", 8 * sum(c["search_entries_nlcc"] for c in every),
                       sum(c["ms_search_kernel"] for c in every), sum(c["search_launches"] for c in every))
    roofline = roof_search if roof_search["device_ms"] > roof_lcc["device_ms"] else roof_lcc
    launches = sum(c["kernel_launches"] for st in agg for c in st.values())

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, ctx, g, cfg, tmpls, stream, local)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        e_cpu, s_cpu, done = cpu_oracle_run(g, cfg["templates"])
        cpu = {"value": e_cpu / s_cpu if s_cpu > 0 else 0.0, "unit": "edges scanned/s", "cores": 1,
               "kind": "oracle", "sample": "whole pipeline, single thread, " + "; ".join(done)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "edges scanned/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic",
                "config": {"workload": args.workload, "graph": f"R-MAT scale {cfg['scale']}, edge factor 16, "
                           f"(.57,.19,.19,.05), {cfg['labels']} labels", "n": g.n, "m_dir": g.m_dir,
                           "templates": {k: {"labels": v[0], "edges": v[1]} for k, v in cfg["templates"].items()},
                           "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}"},
                "tts_ms": tts,
                "search_entries_per_s": search_entries / (total_ms / 1e3) if total_ms > 0 else 0.0,
                "phases": {k: results[k].phase_rounds() for k in tmpls},
                "matches": {k: agg[-1][k]["match_embeddings"] for k in tmpls},
                "roofline": roofline, "rooflines": [roof_lcc, roof_search],
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_e2e(args, ctx, g, cfg, tmpls, stream, local):
    """Same metric through the C ABI from pinned host buffers."""
    import torch
    from paper_1912_08453_gb300 import ccpm
    rp = torch.from_numpy(g.row_ptr).pin_memory()
    col = torch.from_numpy(g.col).pin_memory()
    lab = torch.from_numpy(g.labels).pin_memory()
    words = (g.m_dir + 31) // 32
    outs = {k: (torch.empty(g.n, dtype=torch.int32).pin_memory(),
                torch.empty(words, dtype=torch.int32).pin_memory()) for k in tmpls}
    h2d = rp.numel() * 8 + col.numel() * 4 + lab.numel()
    d2h = len(tmpls) * (g.n * 4 + words * 4)

    def step():
        gr = ccpm.Graph(ctx, rp, col, lab)
        edges = 0
        for k, t in tmpls.items():
            r = ccpm.prune(ctx, gr, t)
            r.omega(outs[k][0])
            r.edge_bitmap(outs[k][1])
            c = r.counts()
            edges += c["edges_scanned_lcc"]
            r.close()
        gr.close()
        return edges

    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            step()
        ms, edges = [], 0
        for _ in range(args.steps):
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            edges += step()
            ev1.record(stream)
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
    return {"value": edges / (sum(ms) / 1e3), "unit": "edges scanned/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": sum(ms) / len(ms)}


if __name__ == "__main__":
    main()
