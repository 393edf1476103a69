#!/usr/bin/env python
"""Benchmark of the constraint-checking pruning pipeline on one GB300.

Headline workload (default, `--workload c4`): many templates over one resident
graph.  R-MAT scale 24 (edge factor 16, (.57,.19,.19,.05)), Zipf(1.2) labels
over 64 labels, generated on the device from seeded Philox draws; 64
templates = a 7-vertex base (a 4-cycle and a triangle sharing an edge, plus a
two-edge tail) and 63 of its edit-distance-1/2 variants (5-9 vertices).

One step = every template of the batch pruned end to end (init, LCC to
fixpoint, every non-local constraint with LCC re-runs, the final
template-driven search that makes omega* and E* exact and counts matches up to
the count cap) with the batched entry point (autotuned) and the learned
constraint order where a check on a slice of the batch finds it faster than
the fixed one.  The same templates are also pruned one at a time in the fixed
order ("plain");
the outputs of the two must be identical (omega words, edge-bitmap words,
match counts), and the line reports both times.

value  = active CSR entries examined by the LCC rounds per second of the
         batched+learned step, device time, inputs resident.  That count is
         the same on every implementation of the method (the GPU path and the
         oracle agree on it entry for entry), so values of different arms
         compare as time ratios.  Entries examined by the searches depend on
         how a search is organised; they are reported beside it
         (`search_entries_per_s`), not in it.
e2e    = the same metric through the C ABI from pinned host buffers: graph
         upload, batched pruning, read-back of every template's omega and
         edge bitmap to the host.
Extras in the same line: the scale-25 single-template configuration (C3,
where omega no longer fits in L2: the LCC roofline case), the scale-22
degree-label configuration (C2), the LCC of a 48-vertex edge-labelled
template (f3, 64-bit omega), rooflines of the LCC round and of the searches,
the CPU oracle timed on the host cores.

Under torchrun each rank prunes a share of the templates (dealt by
warm-up cost, longest first; weak scaling, no collective on the data path);
rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "template time-to-solution (ms) & edges scanned/s, batched+learned vs plain"

C4_BASE = ([20, 30, 40, 20, 50, 60, 30], [(0, 1), (1, 2), (2, 3), (3, 0), (2, 4), (3, 4), (4, 5), (5, 6)])
C3_TEMPLATE = ([20, 30, 40, 20, 30, 50, 60, 40],
               [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (4, 5), (5, 6), (6, 7), (2, 7)])
C3_FREQUENT = ([0, 1, 2, 0, 1, 3, 4, 2], C3_TEMPLATE[1])
TREE6 = ([11, 3, 6, 8, 7, 9], [(0, 1), (1, 2), (1, 3), (3, 4), (4, 5)])
C4TRI6 = ([5, 12, 11, 11, 5, 7], [(0, 1), (1, 2), (2, 3), (3, 0), (2, 4), (3, 4), (4, 5)])

WORKLOADS = {
    # C4: batching over one resident graph (the headline)
    "c4": {"name": "c4-rmat24-zipf-batch64", "scale": 24, "labels": "zipf", "gen": "philox",
           "base": C4_BASE, "batch": 64, "batch_seed": 5},
    # C3: one 8-vertex template with repeated labels and a 5-cycle (TDS) at scale 25
    "c3": {"name": "c3-rmat25-zipf", "scale": 25, "labels": "zipf", "gen": "philox",
           "templates": {"c3_5cycle8": C3_TEMPLATE},
           # the LCC phase of the same template shape over the most frequent
           # labels: about half the vertices start active, so omega (134 MB)
           # is gathered from everywhere (its full pipeline is out of reach:
           # the final step over >10^12 matches)
           "lcc_templates": {"c3_5cycle8_frequent": C3_FREQUENT}},
    # C2: scale 22, degree labels, an LCC-only tree and a 4-cycle + triangle template
    "c2": {"name": "c2-rmat22-degree", "scale": 22, "labels": "degree", "gen": "philox",
           "templates": {"tree6": TREE6, "c4tri6": C4TRI6}},
    # the same two templates on the numpy-generated scale-22 graph (full-size parity test)
    "rmat22-degree": {"name": "rmat22-degree", "scale": 22, "labels": "degree", "gen": "numpy",
                      "templates": {"tree6": TREE6, "c4tri6": C4TRI6}},
    # small cases of the same kernels for profiler captures (a few GB on the
    # device): the C3 template's LCC phase at scale 24, the C4 base template
    # at scale 22
    "c3lcc24": {"name": "c3-lcc-rmat24-zipf", "scale": 24, "labels": "zipf", "gen": "philox",
                "templates": {}, "lcc_templates": {"c3_5cycle8_frequent": C3_FREQUENT}},
    "c4base22": {"name": "c4-base-rmat22-zipf", "scale": 22, "labels": "zipf", "gen": "philox",
                 "templates": {"c4_base": C4_BASE}},
    # f3: LCC for a 48-vertex template with edge labels (64-bit omega words),
    # scale 22, degree labels, three edge labels (weights 8:1:1); the template
    # is a breadth-first sample of the graph itself, so it matches
    "f3": {"name": "f3-wide-rmat22-degree-el3", "scale": 22, "labels": "degree", "gen": "philox",
           "wide": {"n0": 48, "extra": 6, "seed": 48, "n_edge_labels": 3, "weights": [8, 1, 1]}},
    "rmat16-degree": {"name": "rmat16-degree", "scale": 16, "labels": "degree", "gen": "numpy",
                      "templates": {"treetri6": ([5, 4, 8, 7, 4, 5],
                                                 [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)])}},
}

SMI_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ccpm", "reference"], default="ccpm")
    p.add_argument("--workload", default="c4", choices=sorted(WORKLOADS) + ["c5"])
    p.add_argument("--plain-steps", type=int, default=1,
                   help="timed passes of the one-at-a-time fixed-order comparison")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the C2/C3 lines inside the C4 run")
    p.add_argument("--plain-only", action="store_true",
                   help="C4: one plain pass over the batch and nothing else (a profiler's command)")
    p.add_argument("--count-cap", type=int, default=1 << 16,
                   help="matches counted per template before the count is reported invalid "
                        "(omega* and E* stay exact; every C4 template has more than 2^20 matches)")
    return p.parse_args(argv)


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def make_graph(cfg, device=None):
    """The workload's graph: torch tensors on `device` (Philox recipe) or
    numpy arrays (numpy recipe)."""
    from paper_1912_08453_gb300 import workloads as wl
    if cfg["gen"] == "philox":
        return wl.rmat_graph_philox(cfg["scale"], labels=cfg["labels"], device=device or "cpu")
    return wl.rmat_graph(cfg["scale"], labels=cfg["labels"], device=device)


def host_graph(g):
    from paper_1912_08453_gb300 import workloads as wl
    return g.to_host() if isinstance(g, wl.DeviceGraph) else g


def batch_templates(cfg):
    from paper_1912_08453_gb300 import workloads as wl
    tl, te = cfg["base"]
    base = wl.Template(list(tl), list(te), name="base")
    return [base] + wl.edit_variants(base, cfg["batch"] - 1, seed=cfg["batch_seed"], label_pool=sorted(set(tl)))


class ClockSampler:
    """nvidia-smi sampling during the timed region (every 200 ms)."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"ccpm_clocks_{os.getpid()}.csv")

    def start(self):
        try:
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
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        # samples under load: power well above idle
        busy = [r for r in rows if r[2] > 300.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in busy for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in busy), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "samples_under_load": len(busy), "reasons": reasons}


def kernel_source_hash():
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_1912_08453_gb300", "csrc", "ccpm_kernels.cu"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary of
    `workload`, only if it was taken on the current kernel source."""
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


def roofline(kernel, alg_bytes, ms, n_launch, workload, extra=None):
    """Algorithmic bytes over CUDA-event device time, against the measured
    HBM copy bandwidth."""
    peak, kind = measured_peak_hbm()
    achieved = (alg_bytes / 1e9) / (ms / 1e3) if ms > 0 else 0.0
    out = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "peak_source": kind, "traffic": recorded_traffic(kernel, workload),
           "alg_bytes_per_launch": alg_bytes / max(n_launch, 1), "avg_launch_ms": ms / max(n_launch, 1),
           "launches": n_launch, "device_ms": ms}
    if extra:
        out.update(extra)
    return out


def lcc_roofline(counts, workload):
    """k_lcc_round over every round of the given prunes.  Algorithmic bytes
    per round: 8.25 per active entry M_a + 16 per active vertex n_a."""
    return roofline("k_lcc_round", sum(c["lcc_alg_bytes"] for c in counts),
                    sum(c["ms_lcc_kernel"] for c in counts), sum(c["lcc_launches"] for c in counts), workload,
                    {"M_a": sum(c["edges_scanned_lcc"] for c in counts),
                     "n_a": sum(c["lcc_active_vertices"] for c in counts),
                     "R": sum(c["lcc_row_entries"] for c in counts),
                     "kernel_bytes_per_launch": sum(c["lcc_kernel_bytes"] for c in counts) /
                     max(sum(c["lcc_launches"] for c in counts), 1)})


def lcc_first_round(counts):
    """The first LCC round of each prune (all rows of the initially active
    vertices, the costliest round): 8.25 B per active entry."""
    ent = sum(c["lcc_first_entries"] for c in counts)
    ms = sum(c["ms_lcc_first"] for c in counts)
    peak, kind = measured_peak_hbm()
    gbs = (8.25 * ent / 1e9) / (ms / 1e3) if ms > 0 else 0.0
    return {"entries": ent, "ms": ms, "achieved": gbs, "frac": gbs / peak}


def search_roofline(counts, workload):
    """The search kernels (NLCC walks and the final template-driven search):
    8 algorithmic bytes per row entry examined (column index and the
    neighbour's omega); no pass mark (random, combinatorial access).  One
    'launch' here is the search work of one template's prune (the device
    time of its NLCC search passes plus its whole final step), and traffic
    is counted the same way."""
    ent = sum(c["edges_scanned_search"] for c in counts)
    ms = sum(c["ms_search_kernel"] + c["ms_final"] for c in counts)
    return roofline("search kernels per template", 8 * ent, ms, len(counts), workload,
                    {"entries": ent, "note": "per template: k_nlcc_items, k_expand*, k_final_items, k_edge_items, "
                                             "k_edge_search; device time of the NLCC search passes plus the whole "
                                             "final step"})


def cpu_oracle(g_host, templates, parallel):
    """The CPU oracle as it stands on the given templates: (LCC entries,
    seconds, per-template notes, results)."""
    import oracle
    from oracle import pipeline
    oracle.set_parallel(parallel)
    try:
        edges, secs, notes, res = 0, 0.0, [], []
        for name, (tl, te), cap in templates:
            r = pipeline.run(g_host.row_ptr, g_host.col, g_host.labels, tl, te, max_embeddings=cap)
            edges += r.lcc_scanned
            secs += r.seconds
            notes.append(f"{name}: {r.seconds:.1f}s")
            res.append(r)
        return edges, secs, notes, res
    finally:
        oracle.set_parallel(False)


def lscpu_summary():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        keep = [l.split(":", 1)[1].strip() for l in out.splitlines()
                if l.split(":", 1)[0].strip() in ("Model name", "Architecture")]
        return " / ".join(keep)
    except Exception:
        return ""


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, cfg):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    dev = None
    try:
        import torch
        dev = "cuda:0" if torch.cuda.is_available() else None
    except Exception:
        pass
    g = host_graph(make_graph(cfg, device=dev))
    if "base" in cfg:
        # a bounded sample: one template of the batch per step, the variant
        # the oracle finishes fastest (about 7 s on 16 Arm cores), so that
        # the default step counts finish within minutes
        t = batch_templates(cfg)[30]
        sample = [("t30", (t.labels, t.edges), args.count_cap)]
        sample_note = "template t30 of the 64 per step (the variant the oracle finishes fastest), whole pipeline"
    else:
        sample = [(k, v, args.count_cap) for k, v in cfg["templates"].items()]
        sample_note = "every template of the workload per step, whole pipeline"
    times, edges = [], 0
    for _ in range(args.steps):
        e, s, _, _ = cpu_oracle(g, sample, parallel=True)
        edges += e
        times.append(s)
    total = sum(times)
    value = edges / total if total > 0 else 0.0
    cores = oracle.threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "edges scanned/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": cfg["name"], "scale": cfg["scale"], "n": g.n, "m_dir": g.m_dir,
                       "count_cap": args.count_cap},
            "cpu_baseline": {"value": value, "unit": "edges scanned/s", "cores": cores, "kind": "oracle",
                             "sample": sample_note + f" (OpenMP build, {cores} threads; {lscpu_summary()})"},
            "e2e": {"value": value, "unit": "edges scanned/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def timed(stream, fn):
    """(result, CUDA-event ms on `stream`), synchronised on both sides."""
    import torch
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    out = fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    return out, ev0.elapsed_time(ev1)


def same_results(a, b, n, words, device):
    """omega words, edge-bitmap words and match counts equal, compared on the device."""
    import torch
    oa = torch.empty(n, dtype=torch.int32, device=device)
    ob = torch.empty(n, dtype=torch.int32, device=device)
    ea = torch.empty(words, dtype=torch.int32, device=device)
    eb = torch.empty(words, dtype=torch.int32, device=device)
    for x, y in zip(a, b):
        x.omega(oa)
        y.omega(ob)
        x.edge_bitmap(ea)
        y.edge_bitmap(eb)
        cx, cy = x.counts(), y.counts()
        if not (torch.equal(oa, ob) and torch.equal(ea, eb) and cx["match_embeddings"] == cy["match_embeddings"]
                and cx["count_valid"] == cy["count_valid"]):
            return False
    return True


def single_template_line(args, cfg, ctx, stream, local, reps=2):
    """A few plain prunes of each template of a single-template workload:
    time-to-solution and the LCC rooflines (first round and all rounds)."""
    import torch
    from paper_1912_08453_gb300 import ccpm
    t0 = time.time()
    g = make_graph(cfg, device=f"cuda:{local}")
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    cap = ccpm.options(max_embeddings=args.count_cap)
    out = {"workload": cfg["name"], "n": g.n, "m_dir": g.m_dir, "gen_s": gen_s, "templates": {}}
    every = []
    with torch.cuda.stream(stream):
        for name, (tl, te) in cfg["templates"].items():
            t = ccpm.Template(ctx, tl, te)
            r = ccpm.prune(ctx, graph, t, cap, allow_budget=True)       # warm-up (label-grouped rows)
            ms, cs = [], []
            for _ in range(reps):
                r, dt = timed(stream, lambda: ccpm.prune(ctx, graph, t, cap, result=r, allow_budget=True))
                ms.append(dt)
                cs.append(r.counts())
            every += cs
            c = cs[-1]
            out["templates"][name] = {"tts_ms": statistics.median(ms), "phases": r.phase_rounds(),
                                      "matches": c["match_embeddings"], "count_valid": c["count_valid"],
                                      "active_v": c["active_v"], "active_e_dir": c["active_e_dir"],
                                      "ms_lcc": c["ms_lcc"], "ms_nlcc": c["ms_nlcc"], "ms_final": c["ms_final"],
                                      "lcc_first_round": lcc_first_round([c])}
            r.close()
            t.close()
    out["lcc_roofline"] = lcc_roofline(every, cfg["name"])
    out["lcc_first_round"] = lcc_first_round(every)
    # LCC phase alone (options.lcc_only) of the templates kept for it
    lcc_counts = []
    with torch.cuda.stream(stream):
        for name, (tl, te) in cfg.get("lcc_templates", {}).items():
            t = ccpm.Template(ctx, tl, te)
            only = ccpm.options(lcc_only=1)
            r = ccpm.prune(ctx, graph, t, only)
            cs = []
            for _ in range(max(reps, 2)):
                r, dt = timed(stream, lambda: ccpm.prune(ctx, graph, t, only, result=r))
                cs.append(r.counts())
            lcc_counts += cs
            c = cs[-1]
            out["templates"][name + "_lcc_phase"] = {
                "lcc_ms": dt, "rounds": r.phase_rounds(), "active_v_fixpoint": c["active_v"],
                "lcc_first_round": lcc_first_round([c]),
                "lcc_roofline": lcc_roofline([c], cfg["name"] + "-lcc-phase")}
            r.close()
            t.close()
    if lcc_counts:
        out["lcc_phase_roofline"] = lcc_roofline(lcc_counts, cfg["name"] + "-lcc-phase")
        out["lcc_phase_first_round"] = lcc_first_round(lcc_counts)
    graph.close()
    del g
    torch.cuda.empty_cache()
    return out


def wide_line(args, cfg, ctx, stream, local, reps=3):
    """ccpm_lcc_wide on an edge-labelled graph: time, rounds and the roofline.
    Algorithmic bytes per round, by the same accounting as the 32-bit LCC:
    13.25 per active entry (4 column, 8 neighbour omega, 1 edge label, 1/4
    edge bit) and 24 per active vertex (8 offsets, 16 own omega read and
    written)."""
    import torch
    from paper_1912_08453_gb300 import ccpm
    from paper_1912_08453_gb300 import workloads as wl
    t0 = time.time()
    g = make_graph(cfg, device=f"cuda:{local}")
    w = cfg["wide"]
    el = wl.edge_labels(g.row_ptr, g.col, w["n_edge_labels"], seed=w["seed"], weights=w["weights"])
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    h = host_graph(g)
    tl, te, tel = wl.sampled_template(h, el.cpu().numpy(), w["n0"], w["extra"], seed=w["seed"])
    del h
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    graph.set_edge_labels(el)
    ccpm.lcc_wide(ctx, graph, tl, te, tel)              # warm-up
    stats = []
    for _ in range(reps):
        _, _, st = ccpm.lcc_wide(ctx, graph, tl, te, tel)
        stats.append(st)
    st = stats[-1]
    ms = statistics.median(x["ms"] for x in stats)
    alg = 13.25 * st["edges_scanned"] + 24.0 * st["vertices_scanned"]
    out = {"workload": cfg["name"], "n": g.n, "m_dir": g.m_dir, "gen_s": gen_s, "n0": len(tl), "m0": len(te),
           "edge_labels_in_template": len(set(tel)), "ms": ms, "rounds": st["rounds"],
           "active_v_fixpoint": st["active_v"], "active_e_fixpoint": st["active_e_dir"],
           "roofline": roofline("k_wide_round", alg, ms, st["rounds"], cfg["name"],
                                {"M_a": st["edges_scanned"], "n_a": st["vertices_scanned"],
                                 "note": "device time of the whole call (init, rounds, hand-back) per round"})}
    graph.close()
    del g, el
    torch.cuda.empty_cache()
    return out


def run_c4(args, cfg):
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
    dev = f"cuda:{local}"
    t0 = time.time()
    g = make_graph(cfg, device=dev)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    torch.cuda.empty_cache()
    stream = torch.cuda.Stream()
    ctx = ccpm.Context(local, stream=stream.cuda_stream)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    tmpls_all = batch_templates(cfg)
    hs_all = [ccpm.Template(ctx, t.labels, t.edges) for t in tmpls_all]
    cap = ccpm.options(max_embeddings=args.count_cap)
    words = (g.m_dir + 31) // 32

    with torch.cuda.stream(stream):
        # warm-up 1: the plain pipeline over every template; its times deal the
        # templates over the ranks and its logs train the ordering network
        res_all = [None] * len(hs_all)
        for i, h in enumerate(hs_all):
            res_all[i] = ccpm.prune(ctx, graph, h, cap, result=res_all[i], allow_budget=True)
        costs = torch.tensor([r.counts()["ms_total"] for r in res_all], dtype=torch.float64, device=dev)
        if world > 1:
            torch.distributed.broadcast(costs, 0)
        mine = sharding.deal(costs.tolist(), world)[rank]
        hs = [hs_all[i] for i in mine]
        res_plain = [res_all[i] for i in mine]
        recs = [rec for r in res_plain for rec in r.logs()]
        X, y = ordering.targets_from(recs)
        t_train = time.time()
        net = ordering.train(ctx, X, y, steps=2000) if len(recs) >= 8 else None
        train_s = time.time() - t_train
        # the fixed order decides on a slice of this batch whether the learned
        # one is used (plain, one template at a time): only if it is faster
        use_learned, check_fixed, check_learned = (ordering.choose(ctx, graph, hs[:16], net, args.count_cap)
                                                   if net else (False, 0.0, 0.0))
        learned = ordering.learned_options(net, max_embeddings=args.count_cap) if use_learned else cap
        res_batch = ccpm.prune_batch(ctx, graph, hs, learned, allow_budget=True)   # autotunes the workers
        for _ in range(max(args.warmup - 1, 0)):
            ccpm.prune_batch(ctx, graph, hs, learned, results=res_batch, allow_budget=True)

        # timed: K steps of batched + learned order (inputs are larger than L2:
        # the 2.1 GB column array and 67 MB of omega per template)
        if world > 1:
            torch.distributed.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        t_batch, launches, counts_batch = [], 0, []
        for _ in range(args.steps):
            _, ms = timed(stream, lambda: ccpm.prune_batch(ctx, graph, hs, learned, results=res_batch,
                                                           allow_budget=True))
            t_batch.append(ms)
            cs = [r.counts() for r in res_batch]
            launches += sum(c["kernel_launches"] for c in cs)
            counts_batch.append(cs)
        clk = clocks.stop()
        # the comparisons: one template at a time in the fixed order (plain),
        # batched in the fixed order, and one at a time in the learned order
        t_plain, counts_plain = [], []
        for _ in range(args.plain_steps):
            def plain():
                for i, h in enumerate(hs):
                    res_plain[i] = ccpm.prune(ctx, graph, h, cap, result=res_plain[i], allow_budget=True)
            _, ms = timed(stream, plain)
            t_plain.append(ms)
            counts_plain = [r.counts() for r in res_plain]
        res_bfix = ccpm.prune_batch(ctx, graph, hs, cap, allow_budget=True)
        _, ms_bfix = timed(stream, lambda: ccpm.prune_batch(ctx, graph, hs, cap, results=res_bfix, allow_budget=True))
        res_plearn = [None] * len(hs)

        always_learned = ordering.learned_options(net, max_embeddings=args.count_cap) if net else cap

        def plain_learned():
            for i, h in enumerate(hs):
                res_plearn[i] = ccpm.prune(ctx, graph, h, always_learned, result=res_plearn[i], allow_budget=True)
        _, ms_plearn = timed(stream, plain_learned)
        # ablation (Sec. 6.6): the plain pass again without edge elimination
        abl = ccpm.options(max_embeddings=args.count_cap, no_edge_elimination=1)
        res_abl = [None] * len(hs)

        def plain_no_eta():
            for i, h in enumerate(hs):
                res_abl[i] = ccpm.prune(ctx, graph, h, abl, result=res_abl[i], allow_budget=True)
        plain_no_eta()
        _, ms_abl = timed(stream, plain_no_eta)
        same_abl = same_results(res_plain, res_abl, g.n, words, dev)
        for r in res_abl:
            r.close()
        same = same_results(res_plain, res_batch, g.n, words, dev) and \
            same_results(res_plain, res_bfix, g.n, words, dev) and \
            same_results(res_plain, res_plearn, g.n, words, dev)
        nlcc_plain = sum(c["ms_nlcc"] for c in counts_plain)
        nlcc_plearn = sum(r.counts()["ms_nlcc"] for r in res_plearn)

    edges = sum(c["edges_scanned_lcc"] for cs in counts_batch for c in cs)
    search_entries = sum(c["edges_scanned_search"] for cs in counts_batch for c in cs)
    total_ms = sum(t_batch)
    ms_plain = statistics.median(t_plain)
    total_ms, edges, same = sharding.reduce_step(total_ms, edges, same, device=dev)
    ms_plain, _, _ = sharding.reduce_step(ms_plain, 0, True, device=dev)

    e2e = None
    if not args.no_e2e and world == 1:
        # every e2e step loads the graph anew: it runs with the settings the
        # autotuner chose on the resident graph (a user keeps them the same way)
        tune = ccpm.batch_tuning(graph)
        e2e_opt = ccpm.Options.from_buffer_copy(learned)
        e2e_opt.batch_workers = tune["workers"]
        e2e_opt.grid_share = tune["grid_share"]
        e2e_opt.search_split = tune["search_split"]
        e2e_opt.short_rows = tune["short_rows"]
        e2e_opt.hub_degree = tune["hub_degree"]
        e2e = run_c4_e2e(args, ctx, g, hs, e2e_opt, stream)

    cpu = None
    oracle_parity = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, oracle_parity = c4_cpu_baseline(args, g, tmpls_all, counts_plain, res_plain, mine, dev)

    # rooflines from the plain pass (every kernel runs alone on the stream)
    roof_lcc = lcc_roofline(counts_plain, cfg["name"])
    roof_search = search_roofline(counts_plain, cfg["name"])
    dominant = roof_search if roof_search["device_ms"] > roof_lcc["device_ms"] else roof_lcc
    workers = ccpm.batch_tuning(graph)
    n_graph, m_graph = int(graph.n), int(graph.m)
    for r in res_all + res_batch + res_bfix + res_plearn:
        if r is not None:
            r.close()

    graph.close()
    del g
    torch.cuda.empty_cache()
    extras = {}
    if not args.no_extras and world == 1:
        extras["c3"] = single_template_line(args, WORKLOADS["c3"], ctx, stream, local)
        extras["c2"] = single_template_line(args, WORKLOADS["c2"], ctx, stream, local, reps=3)
        extras["f3"] = wide_line(args, WORKLOADS["f3"], ctx, stream, local)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    value = edges / (total_ms / 1e3) if total_ms > 0 else 0.0
    tts = [c["ms_total"] for c in counts_batch[-1]]
    line = {"metric": METRIC, "value": value, "unit": "edges scanned/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": cfg["name"],
                       "graph": f"R-MAT scale {cfg['scale']}, edge factor 16, (.57,.19,.19,.05), "
                                "Zipf(1.2) labels over 64, Philox-generated on the device",
                       "n": n_graph, "m_dir": m_graph, "templates": len(hs_all),
                       "templates_rank0": len(hs), "template_sizes": sorted({t.n0 for t in tmpls_all}),
                       "base_template": {"labels": cfg["base"][0], "edges": cfg["base"][1]},
                       "count_cap": args.count_cap,
                       "l2": "inputs larger than L2 (2.1 GB column array), no flush",
                       "parallelism": f"templates dealt over {world} ranks" if world > 1 else "one GPU"},
            "plain_ms": ms_plain, "batched_learned_ms": total_ms / args.steps,
            "batched_step_ms": t_batch,
            "speedup": ms_plain / (total_ms / args.steps) if total_ms > 0 else None,
            "batched_fixed_ms": ms_bfix, "plain_learned_ms": ms_plearn,
            "nlcc_ms_plain_fixed": nlcc_plain, "nlcc_ms_plain_learned": nlcc_plearn,
            "identical_outputs": bool(same),
            "ablation_edge_elimination": {"plain_ms_without": ms_abl, "plain_ms_with": ms_plain,
                                          "slowdown_without": ms_abl / ms_plain if ms_plain else None,
                                          "identical_outputs": bool(same_abl),
                                          "paper": "2-9x faster with edge elimination (Sec. 6.6, WDC-3)"},
            "tts_ms": {"median": statistics.median(tts), "max": max(tts), "sum": sum(tts)},
            "plain_split_ms": {k: sum(c[k] for c in counts_plain) for k in
                               ("ms_lcc", "ms_nlcc", "ms_final", "ms_final_count", "ms_final_vertex",
                                "ms_final_edge")},
            "counts_valid": int(sum(c["count_valid"] for c in counts_plain)),
            "autotune": workers,
            "training_records": len(recs), "training_s": train_s, "graph_gen_s": gen_s,
            "learned_order": {"used_in_batch": bool(use_learned), "check_slice_ms_fixed": check_fixed,
                              "check_slice_ms_learned": check_learned,
                              "note": "the learned order is used only if faster than the fixed one on the first 16 templates; "
                                      "plain_learned_ms always uses the learned order"},
            "search_entries_per_s": search_entries / (total_ms / 1e3) if total_ms > 0 else 0.0,
            "roofline": dominant, "rooflines": [roof_lcc, roof_search],
            "lcc_first_round": lcc_first_round(counts_plain),
            "cpu_baseline": cpu, "oracle_parity_sample": oracle_parity, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches}
    line.update(extras)
    print(json.dumps(line), flush=True)


def run_c4_e2e(args, ctx, g, hs, learned, stream):
    """The headline through the C ABI from pinned host buffers: the graph is
    uploaded every step, the batch pruned, and every template's omega and edge
    bitmap read back into pinned host memory."""
    import torch
    from paper_1912_08453_gb300 import ccpm
    rp = g.row_ptr.cpu().pin_memory()
    col = g.col.cpu().pin_memory()
    lab = g.labels.cpu().pin_memory()
    words = (g.m_dir + 31) // 32
    om_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
    eb_h = torch.empty(words, dtype=torch.int32).pin_memory()
    h2d = rp.numel() * 8 + col.numel() * 4 + lab.numel()
    d2h = len(hs) * (g.n * 4 + words * 4)

    def step():
        gr = ccpm.Graph(ctx, rp, col, lab)
        res = ccpm.prune_batch(ctx, gr, hs, learned, allow_budget=True)
        edges = 0
        for r in res:
            r.omega(om_h)
            r.edge_bitmap(eb_h)
            edges += r.counts()["edges_scanned_lcc"]
            r.close()
        gr.close()
        return edges

    with torch.cuda.stream(stream):
        step()
        ms, edges = [], 0
        for _ in range(max(1, min(args.steps, 2))):
            e, dt = timed(stream, step)
            edges += e
            ms.append(dt)
    return {"value": edges / (sum(ms) / 1e3), "unit": "edges scanned/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": sum(ms) / len(ms), "steps": len(ms)}


def c4_cpu_baseline(args, g, tmpls_all, counts_plain, res_plain, mine, dev):
    """The oracle on a bounded sample of the batch (the templates the GPU
    pruned fastest, so the sample stays within tens of seconds), single
    threaded and with OpenMP on every host core; the sample's GPU results are
    checked against it entry for entry."""
    import oracle
    oracle.build()
    gh = host_graph(g)
    order = sorted(range(len(counts_plain)), key=lambda i: counts_plain[i]["ms_total"])
    pick = order[:2]
    sample = [(f"t{mine[i]}", (tmpls_all[mine[i]].labels, tmpls_all[mine[i]].edges), args.count_cap) for i in pick]
    e1, s1, n1, ref1 = cpu_oracle(gh, sample[:1], parallel=False)
    e2, s2, n2, ref2 = cpu_oracle(gh, sample, parallel=True)
    parity = True
    for i, ref in zip(pick, ref2):
        r = res_plain[i]
        parity &= bool(np.array_equal(r.omega(), ref.omega) and np.array_equal(r.edge_bitmap(), ref.ebits)
                       and r.phase_rounds() == ref.phase_rounds
                       and r.counts()["match_embeddings"] == ref.match_embeddings)
    cores = oracle.threads()
    cpu = {"value": e2 / s2 if s2 > 0 else 0.0, "unit": "edges scanned/s", "cores": cores, "kind": "oracle",
           "sample": f"{len(sample)} of the 64 templates (those the GPU pruned fastest), whole pipeline, "
                     f"OpenMP build: " + "; ".join(n2) + f" ({lscpu_summary()})",
           "single_thread": {"value": e1 / s1 if s1 > 0 else 0.0, "cores": 1, "sample": "; ".join(n1)}}
    return cpu, {"templates": [s[0] for s in sample], "identical": parity}


def c5_training_templates(count, seed, label_pool):
    """Random connected templates (4-9 vertices, 0-3 chords, labels with
    repeats from a small per-template subset of `label_pool`)."""
    from paper_1912_08453_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n0 = int(rng.integers(4, 10))
        extra = int(rng.integers(0, 4))
        pool = [int(x) for x in rng.choice(label_pool, size=int(rng.integers(2, 5)), replace=False)]
        out.append(wl.random_template(seed * 100003 + i, n0, extra, pool))
    return out


def c5_eval_templates(seed, label_pool):
    """32 evaluation templates: 12 four-cycles, 10 five-cycles, 10 four-cliques."""
    from paper_1912_08453_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    shapes = ([("c4", 4, [(0, 1), (1, 2), (2, 3), (3, 0)])] * 12 +
              [("c5", 5, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)])] * 10 +
              [("k4", 4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])] * 10)
    out = []
    for i, (kind, n0, edges) in enumerate(shapes):
        labels = [int(x) for x in rng.choice(label_pool, size=n0)]
        out.append(wl.Template(labels, edges, name=f"{kind}-{i}"))
    return out


def run_c5(args):
    """Learned constraint ordering at its stated scale: logs of the plain
    pipeline over 2,000 random templates on scale-20 graphs train the network
    (on the GPU, with the library's kernels); 32 templates (4-/5-cycles,
    4-cliques) on a scale-25 graph are then pruned in the fixed and in the
    learned order.  Outputs must be identical; times are compared."""
    import torch
    from paper_1912_08453_gb300.build import build
    from paper_1912_08453_gb300 import ccpm, ordering
    from paper_1912_08453_gb300 import workloads as wl
    build()
    dev = "cuda:0"
    stream = torch.cuda.Stream()
    ctx = ccpm.Context(0, stream=stream.cuda_stream)
    tail = list(range(16, 64))
    t0 = time.time()
    recs, n_tmpl = [], 0
    per_graph = 2000 // 3
    with torch.cuda.stream(stream):
        for gi, gseed in enumerate((11, 12, 13)):
            g = wl.rmat_graph_philox(20, labels="zipf", seed=gseed, label_seed=gseed + 100, device=dev)
            graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
            count = per_graph + (2000 - 3 * per_graph if gi == 2 else 0)
            for t in c5_training_templates(count, gseed, tail):
                h = ccpm.Template(ctx, t.labels, t.edges)
                r = ccpm.prune(ctx, graph, h, ccpm.options(run_final=0), allow_budget=True)
                recs += r.logs()
                n_tmpl += 1
                r.close()
                h.close()
            graph.close()
            del g
            torch.cuda.empty_cache()
    collect_s = time.time() - t0
    X, y = ordering.targets_from(recs)
    t1 = time.time()
    net = ordering.train(ctx, X, y, steps=4000)
    train_s = time.time() - t1
    learned = ordering.learned_options(net, max_embeddings=args.count_cap)
    fixed = ccpm.options(max_embeddings=args.count_cap)
    g = wl.rmat_graph_philox(25, labels="zipf", device=dev)
    torch.cuda.synchronize()
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    words = (g.m_dir + 31) // 32
    rows = []
    with torch.cuda.stream(stream):
        for t in c5_eval_templates(5, tail):
            h = ccpm.Template(ctx, t.labels, t.edges)
            nc = h.generate()
            r_f = ccpm.prune(ctx, graph, h, fixed, allow_budget=True)        # warm-up
            r_f, ms_f = timed(stream, lambda: ccpm.prune(ctx, graph, h, fixed, result=r_f, allow_budget=True))
            r_l = ccpm.prune(ctx, graph, h, learned, allow_budget=True)
            r_l, ms_l = timed(stream, lambda: ccpm.prune(ctx, graph, h, learned, result=r_l, allow_budget=True))
            same = same_results([r_f], [r_l], g.n, words, dev)
            cf, cl = r_f.counts(), r_l.counts()
            rows.append({"template": t.name, "constraints": nc, "identical": same, "ms_fixed": ms_f,
                         "ms_learned": ms_l, "nlcc_ms_fixed": cf["ms_nlcc"], "nlcc_ms_learned": cl["ms_nlcc"],
                         "order_changed": r_f.order() != r_l.order()})
            r_f.close()
            r_l.close()
            h.close()
    fam = {}
    for kind in ("c4", "c5", "k4"):
        sel = [r for r in rows if r["template"].startswith(kind)]
        fam[kind] = {"templates": len(sel), "ms_fixed": sum(r["ms_fixed"] for r in sel),
                     "ms_learned": sum(r["ms_learned"] for r in sel),
                     "nlcc_ms_fixed": sum(r["nlcc_ms_fixed"] for r in sel),
                     "nlcc_ms_learned": sum(r["nlcc_ms_learned"] for r in sel),
                     "orders_changed": sum(r["order_changed"] for r in sel)}
    tot_f = sum(r["ms_fixed"] for r in rows)
    tot_l = sum(r["ms_learned"] for r in rows)
    line = {"workload": "c5-learned-ordering", "training_templates": n_tmpl, "training_records": len(recs),
            "collect_s": collect_s, "train_s": train_s, "eval_graph": f"R-MAT scale 25, n={g.n}, m={g.m_dir}",
            "identical_outputs": all(r["identical"] for r in rows), "ms_fixed": tot_f, "ms_learned": tot_l,
            "gain": tot_f / tot_l if tot_l else None,
            "nlcc_gain": (sum(r["nlcc_ms_fixed"] for r in rows) / max(sum(r["nlcc_ms_learned"] for r in rows), 1e-9)),
            "families": fam, "rows": rows}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.workload == "c5":
        run_c5(args)
        return
    cfg = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, cfg)
        return
    if "base" in cfg and args.plain_only:
        run_c4_plain_pass(args, cfg)
        return
    if "base" in cfg:
        run_c4(args, cfg)
        return
    run_single(args, cfg)


def run_c4_plain_pass(args, cfg):
    """One plain pass over the batch (one template at a time, fixed order):
    the command the search kernels' DRAM counters are taken on, so that they
    divide by exactly the templates of one pass."""
    import torch
    from paper_1912_08453_gb300.build import build
    from paper_1912_08453_gb300 import ccpm
    build()
    g = make_graph(cfg, device="cuda:0")
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    ctx = ccpm.Context(0, stream=stream.cuda_stream)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    cap = ccpm.options(max_embeddings=args.count_cap)
    hs = [ccpm.Template(ctx, t.labels, t.edges) for t in batch_templates(cfg)]
    with torch.cuda.stream(stream):
        res = []
        for h in hs:
            res.append(ccpm.prune(ctx, graph, h, cap, allow_budget=True))
    counts = [r.counts() for r in res]
    print(json.dumps({"workload": cfg["name"] + "-plain-pass", "templates": len(hs),
                      "search_entries": sum(c["edges_scanned_search"] for c in counts),
                      "search_device_ms": sum(c["ms_search_kernel"] + c["ms_final"] for c in counts),
                      "lcc_launches": sum(c["lcc_launches"] for c in counts),
                      "lcc_alg_bytes": sum(c["lcc_alg_bytes"] for c in counts)}), flush=True)


def run_single(args, cfg):
    """A single-template workload on its own (C2, C3, C1): plain prunes."""
    import torch
    from paper_1912_08453_gb300.build import build
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if rank == 0:
        build()
    from paper_1912_08453_gb300 import ccpm
    stream = torch.cuda.Stream()
    ctx = ccpm.Context(local, stream=stream.cuda_stream)
    clocks = ClockSampler(local)
    clocks.start()
    if "wide" in cfg:
        out = wide_line(args, cfg, ctx, stream, local, reps=max(args.steps, 1))
        clk = clocks.stop()
        if rank != 0:
            return
        roof = out["roofline"]
        line = {"metric": METRIC, "value": roof["M_a"] / (out["ms"] / 1e3) if out["ms"] else 0.0,
                "unit": "edges scanned/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": out["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u64", "data": "synthetic", "config": {"workload": cfg["name"], "n": out["n"],
                                                                "m_dir": out["m_dir"]},
                "roofline": roof, "detail": out, "clocks": clk, "cpu_baseline": None, "e2e": None,
                "gpu_launches": None}
        print(json.dumps(line), flush=True)
        return
    out = single_template_line(args, cfg, ctx, stream, local, reps=max(args.steps, 1))
    clk = clocks.stop()
    if rank != 0:
        return
    tts = sum(v.get("tts_ms", v.get("lcc_ms", 0.0)) for v in out["templates"].values())
    roof = out["lcc_roofline"] if cfg["templates"] else out.get("lcc_phase_roofline", out["lcc_roofline"])
    line = {"metric": METRIC, "value": roof["M_a"] / max(args.steps, 1) / (tts / 1e3) if tts else 0.0,
            "unit": "edges scanned/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tts, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic", "config": {"workload": cfg["name"], "n": out["n"],
                                                            "m_dir": out["m_dir"]},
            "roofline": roof, "detail": out, "clocks": clk, "cpu_baseline": None, "e2e": None,
            "gpu_launches": None}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
