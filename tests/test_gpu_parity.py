"""GPU path vs oracle, element by element, through the C ABI.

Bit-exact on every integer output: omega words, edge-bitmap words, LCC rounds
per phase, match count, tokens issued, active entries scanned by LCC.
"""
import json
import os

import numpy as np
import pytest

from paper_1912_08453_gb300 import workloads as wl
from oracle import pipeline

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    from paper_1912_08453_gb300 import ccpm
    return ccpm.Context(0)


def gpu_run(ctx, g, tl, te, **opt):
    from paper_1912_08453_gb300 import ccpm
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    t = ccpm.Template(ctx, tl, te)
    r = ccpm.prune(ctx, graph, t, ccpm.options(**opt), allow_budget=True)
    out = dict(omega=r.omega(), ebits=r.edge_bitmap(), counts=r.counts(), phases=r.phase_rounds())
    r.close()
    t.close()
    graph.close()
    return out


def assert_parity(ctx, g, tl, te, **opt):
    gpu = gpu_run(ctx, g, tl, te, **opt)
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    np.testing.assert_array_equal(gpu["omega"], ref.omega)
    np.testing.assert_array_equal(gpu["ebits"], ref.ebits)
    assert gpu["phases"] == ref.phase_rounds
    c = gpu["counts"]
    assert c["count_valid"] == int(ref.count_valid)
    assert c["match_embeddings"] == ref.match_embeddings
    assert c["edges_scanned_lcc"] == ref.lcc_scanned
    assert c["tokens"] == ref.tokens
    assert c["active_v"] == ref.active_v
    assert c["active_e_dir"] == ref.active_e_dir
    assert c["automorphisms"] == ref.automorphisms
    return gpu, ref


def random_graph(seed, n, p, n_labels):
    rng = np.random.default_rng(seed)
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
    return wl.graph_from_edge_list(n, edges, rng.integers(0, n_labels, size=n))


TEMPLATES = [
    ([0, 1, 2], [(0, 1), (1, 2), (0, 2)]),
    ([0, 0, 1], [(0, 1), (1, 2), (0, 2)]),
    ([0, 1, 2, 0], [(0, 1), (1, 2), (2, 3)]),
    ([0, 1, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 0)]),
    ([0, 1, 1, 1], [(0, 1), (0, 2), (0, 3)]),
    ([0, 1, 2, 0], [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
    ([0, 1, 2, 0, 1], [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3), (0, 4), (1, 4), (2, 4)]),
    ([0, 1, 2, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)]),
    ([2, 0, 1, 0, 2], [(0, 1), (1, 2), (2, 3), (3, 4)]),
]


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("ti", range(len(TEMPLATES)))
def test_tiny_random(ctx, seed, ti):
    tl, te = TEMPLATES[ti]
    g = random_graph(50 + seed, 24, 0.3, max(tl) + 1)
    assert_parity(ctx, g, tl, te)


def test_fig2_fixtures(ctx):
    for name in ("fig2a_cycle9.json", "fig2c_torus.json"):
        fx = json.load(open(os.path.join(GOLDEN, name)))
        gd = fx["graph"]
        g = wl.graph_from_edge_list(gd["n"], gd["edges"], gd["labels"])
        gpu, ref = assert_parity(ctx, g, fx["template"]["labels"],
                                 [tuple(e) for e in fx["template"]["edges"]])
        assert gpu["counts"]["match_embeddings"] == fx["expect"]["matches"]


def test_rmat16_tree_triangle(ctx):
    # workload C1: R-MAT scale 16, degree labels, 6-vertex tree + triangle
    g = wl.rmat_graph(16)
    gpu, ref = assert_parity(ctx, g, [5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)])
    assert ref.match_embeddings > 0 and len(ref.phase_rounds) == 4


@pytest.mark.parametrize("seed", range(6))
def test_rmat14_random_templates(ctx, seed):
    g = wl.rmat_graph(14, seed=seed + 10)
    pool = [L for L in wl.labels_by_frequency(g) if L > 0][:6]
    t = wl.random_template(seed, 4 + seed % 4, seed % 3, pool)
    assert_parity(ctx, g, t.labels, t.edges)


def test_split_rows_path(ctx):
    # hub rows split into pieces of 8 entries: exercises the combined path
    g = wl.rmat_graph(13, seed=5)
    assert_parity(ctx, g, [5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)],
                  hub_degree=8)
    g.labels = np.zeros(g.n, dtype=np.uint8)
    assert_parity(ctx, g, [0, 0, 0], [(0, 1), (1, 2), (0, 2)], hub_degree=16)


def test_many_classes_path(ctx):
    # unlabelled K5: every vertex has a 4-neighbour class -> 5 classes (wide path)
    g = random_graph(9, 30, 0.5, 1)
    k5 = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    assert_parity(ctx, g, [0] * 5, k5)


def test_unlabelled_closed_form_counts(ctx):
    g = wl.rmat_graph(9, seed=2)
    g.labels = np.zeros(g.n, dtype=np.uint8)
    M = np.zeros((g.n, g.n), dtype=np.int64)
    for v in range(g.n):
        M[v, g.col[g.row_ptr[v]:g.row_ptr[v + 1]]] = 1
    gpu = gpu_run(ctx, g, [0, 0, 0], [(0, 1), (1, 2), (0, 2)])
    assert gpu["counts"]["match_embeddings"] == int(np.trace(M @ M @ M))


def test_edge_cases(ctx):
    # single vertex, no edges
    g = wl.Graph(1, np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(1, dtype=np.uint8))
    gpu = gpu_run(ctx, g, [0, 0], [(0, 1)])
    assert gpu["counts"]["active_v"] == 0 and gpu["counts"]["match_embeddings"] == 0
    # template labels absent from the graph; isolated vertices present
    g = random_graph(3, 40, 0.05, 2)
    assert_parity(ctx, g, [7, 8, 9], [(0, 1), (1, 2)])
    # ragged entry count (not a multiple of 32) and an edge-only graph
    g = wl.graph_from_edge_list(3, [(0, 1), (1, 2)], [0, 1, 0])
    assert g.m_dir % 32 != 0
    assert_parity(ctx, g, [0, 1, 0], [(0, 1), (1, 2)])


def test_without_final_search(ctx):
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph(14, seed=4)
    tl, te = [5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)]
    gpu = gpu_run(ctx, g, tl, te, run_final=0)
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    np.testing.assert_array_equal(gpu["omega"], ref.omega_pre_final)
    from oracle import pack_bits
    np.testing.assert_array_equal(gpu["ebits"], pack_bits(ref.A_pre_final))


def test_deterministic_and_result_reuse(ctx):
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph(14, seed=8)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    t = ccpm.Template(ctx, [5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)])
    r = ccpm.prune(ctx, graph, t)
    a = (r.omega().copy(), r.edge_bitmap().copy(), r.phase_rounds())
    ccpm.prune(ctx, graph, t, result=r)
    b = (r.omega(), r.edge_bitmap(), r.phase_rounds())
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[2] == b[2]


def test_device_pointer_graph(ctx):
    import torch
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph(12, seed=6)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    lab = torch.from_numpy(g.labels).cuda()
    graph = ccpm.Graph(ctx, rp, col, lab)
    tl, te = [5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)]
    t = ccpm.Template(ctx, tl, te)
    r = ccpm.prune(ctx, graph, t)
    om = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    r.omega(om)
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    np.testing.assert_array_equal(om.cpu().numpy().view(np.uint32), ref.omega)


def test_full_size_rmat22_workload(ctx):
    # the benchmark workload at full size (R-MAT scale 22, degree labels), in
    # the same launch configuration the benchmark times
    import bench
    cfg = bench.WORKLOADS["rmat22-degree"]
    g = wl.rmat_graph(cfg["scale"], labels=cfg["labels"])
    for name, (tl, te) in cfg["templates"].items():
        gpu, ref = assert_parity(ctx, g, tl, te)
        assert ref.match_embeddings > 0, name


def test_batch_equals_one_at_a_time(ctx):
    # the batched entry point gives each template exactly its own prune
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph(14, seed=12)
    pool = [L for L in wl.labels_by_frequency(g) if L > 0][:6]
    base = wl.Template([5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)])
    tmpls = [base] + wl.edit_variants(base, 11, seed=3, label_pool=pool, n_min=4, n_max=8)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    hs = [ccpm.Template(ctx, t.labels, t.edges) for t in tmpls]
    # autotuned; then three workers whose grids use a quarter of the SMs each
    for workers, share in ((0, 0), (3, 4)):
        res = ccpm.prune_batch(ctx, graph, hs, ccpm.options(batch_workers=workers, grid_share=share))
        if workers == 0:
            # the autotuner chose and recorded every setting it tunes
            tune = ccpm.batch_tuning(graph)
            assert tune["workers"] in (1, 2, 4, 8, 16) and tune["grid_share"] in (1, 2, 4)
            assert tune["search_split"] in (0, 512, 8192)
            assert tune["short_rows"] in (0, 32, 256) and tune["hub_degree"] in (0, 4096)
            assert tune["slice_ms"] > 0
        for t, h, r in zip(tmpls, hs, res):
            one = ccpm.prune(ctx, graph, h)
            np.testing.assert_array_equal(r.omega(), one.omega())
            np.testing.assert_array_equal(r.edge_bitmap(), one.edge_bitmap())
            assert r.phase_rounds() == one.phase_rounds()
            assert r.counts()["match_embeddings"] == one.counts()["match_embeddings"]
            one.close()
        for r in res:
            r.close()
    # and every result also equals the oracle
    for t, h in zip(tmpls[:4], hs[:4]):
        r = ccpm.prune_batch(ctx, graph, [h])[0]
        ref = pipeline.run(g.row_ptr, g.col, g.labels, t.labels, t.edges)
        np.testing.assert_array_equal(r.omega(), ref.omega)
        np.testing.assert_array_equal(r.edge_bitmap(), ref.ebits)


def test_count_cap_keeps_exact_sets(ctx):
    # past max_embeddings the count is reported invalid; omega* and E* stay exact
    g = wl.rmat_graph(12, seed=7)
    g.labels = (np.arange(g.n) % 2).astype(np.uint8)
    tl, te = [0, 1, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 0)]
    ref_full = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    assert ref_full.match_embeddings > 10
    gpu = gpu_run(ctx, g, tl, te, max_embeddings=10)
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te, max_embeddings=10)
    assert gpu["counts"]["count_valid"] == 0 and not ref.count_valid
    np.testing.assert_array_equal(gpu["omega"], ref.omega)
    np.testing.assert_array_equal(gpu["ebits"], ref.ebits)
    np.testing.assert_array_equal(ref.omega, ref_full.omega)


def test_edge_elimination_ablation_keeps_the_result(ctx):
    # options.no_edge_elimination: LCC counts every live neighbour, so its
    # fixpoint is larger (more rounds of work later), but the final exact
    # search gives the same omega*, E* and count as the method (Sec. 6.6's
    # ablation measures only the time)
    g = wl.rmat_graph(14, seed=10)
    pool = [L for L in wl.labels_by_frequency(g) if L > 0][:6]
    base = wl.Template([5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)])
    for t in [base] + wl.edit_variants(base, 5, seed=9, label_pool=pool, n_min=4, n_max=8):
        on = gpu_run(ctx, g, t.labels, t.edges)
        off = gpu_run(ctx, g, t.labels, t.edges, no_edge_elimination=1)
        np.testing.assert_array_equal(on["omega"], off["omega"])
        np.testing.assert_array_equal(on["ebits"], off["ebits"])
        assert on["counts"]["match_embeddings"] == off["counts"]["match_embeddings"]


def test_entry_label_first_round(ctx):
    # options.entry_labels: the first round reads the per-graph copy of the
    # neighbour labels in entry order instead of the column index and the
    # label gather; the whole pipeline stays oracle-exact, on the short-row,
    # warp-per-row and split-row paths, with and without the final search
    g = wl.rmat_graph(14, seed=12)
    tl, te = [5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)]
    for opt in (dict(entry_labels=1), dict(entry_labels=1, hub_degree=8, short_rows=4)):
        assert_parity(ctx, g, tl, te, **opt)
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    from oracle import pack_bits
    for el in (1, -1):
        gpu = gpu_run(ctx, g, tl, te, entry_labels=el, run_final=0)
        np.testing.assert_array_equal(gpu["omega"], ref.omega_pre_final)
        np.testing.assert_array_equal(gpu["ebits"], pack_bits(ref.A_pre_final))
    # the first LCC fixpoint alone (every round on the full rows): the live
    # rows are exact after the quiescent round, the dead rows are zeroed
    g.labels = np.zeros(g.n, dtype=np.uint8)
    g.labels[::3] = 1
    tl2, te2 = [0, 1, 0, 0], [(0, 1), (1, 2), (2, 3), (3, 0)]
    import oracle
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om_o, A_o = oracle.init(og, tl2, te2)
    rounds, scanned = oracle.lcc(og, tl2, te2, om_o, A_o)
    assert np.count_nonzero(om_o) > 0
    for el in (1, -1):
        for comp in (-1, 1):
            gpu = gpu_run(ctx, g, tl2, te2, entry_labels=el, lcc_only=1, compact=comp)
            assert gpu["phases"] == [rounds]
            assert gpu["counts"]["edges_scanned_lcc"] == scanned
            np.testing.assert_array_equal(gpu["omega"], om_o)
            np.testing.assert_array_equal(gpu["ebits"], oracle.pack_bits(A_o))
