"""Row compaction between LCC rounds (frontier and edge-bitmap compaction):
the compacted pipeline must give the oracle's results bit for bit -- omega,
edge bitmap, LCC rounds per phase, active entries scanned, tokens and match
counts -- whether it compacts after every round, automatically, or never.
"""
import numpy as np
import pytest

from paper_1912_08453_gb300 import workloads as wl
from oracle import pipeline

pytestmark = pytest.mark.gpu

TEMPLATES = {
    "treetri6": ([5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)]),
    "c4p6": ([7, 8, 7, 4, 4, 6], [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 5)]),
    "tree5": ([6, 4, 5, 7, 4], [(0, 1), (1, 2), (1, 3), (3, 4)]),
    "tri_rep": ([5, 5, 6], [(0, 1), (1, 2), (0, 2)]),
}


@pytest.fixture(scope="module")
def env():
    from paper_1912_08453_gb300 import ccpm
    ctx = ccpm.Context(0)
    g = wl.rmat_graph(16, labels="degree")
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    yield ccpm, ctx, g, graph
    graph.close()
    ctx.close()


def run(ccpm, ctx, graph, tl, te, **opt):
    t = ccpm.Template(ctx, tl, te)
    r = ccpm.prune(ctx, graph, t, ccpm.options(**opt), allow_budget=True)
    out = dict(omega=r.omega(), ebits=r.edge_bitmap(), counts=r.counts(), phases=r.phase_rounds())
    r.close()
    t.close()
    return out


def check(out, ref, final=True):
    np.testing.assert_array_equal(out["omega"], ref.omega if final else ref.omega_pre_final)
    if final:
        np.testing.assert_array_equal(out["ebits"], ref.ebits)
        assert out["counts"]["match_embeddings"] == ref.match_embeddings
        assert out["counts"]["count_valid"] == int(ref.count_valid)
    assert out["phases"] == ref.phase_rounds
    assert out["counts"]["edges_scanned_lcc"] == ref.lcc_scanned
    assert out["counts"]["tokens"] == ref.tokens


@pytest.mark.parametrize("name", sorted(TEMPLATES))
@pytest.mark.parametrize("mode", [1, 0, -1])
@pytest.mark.parametrize("hub", [0, 8])
def test_compaction_parity(env, name, mode, hub):
    ccpm, ctx, g, graph = env
    tl, te = TEMPLATES[name]
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    out = run(ccpm, ctx, graph, tl, te, compact=mode, hub_degree=hub)
    check(out, ref)
    if mode == 1 and ref.lcc_rounds_total > 2:
        assert out["counts"]["lcc_compactions"] > 0
    if mode == -1:
        assert out["counts"]["lcc_compactions"] == 0


@pytest.mark.parametrize("name", sorted(TEMPLATES))
def test_compaction_without_final(env, name):
    """Edge map handed back from the LCC/NLCC state (no final search): the
    fixpoint form of the bitmap equals the oracle's Jacobi state."""
    ccpm, ctx, g, graph = env
    tl, te = TEMPLATES[name]
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    for mode in (1, -1):
        out = run(ccpm, ctx, graph, tl, te, compact=mode, run_final=0)
        np.testing.assert_array_equal(out["omega"], ref.omega_pre_final)
        np.testing.assert_array_equal(out["ebits"], wl_pack(ref.A_pre_final))
        assert out["phases"] == ref.phase_rounds


def wl_pack(A):
    from oracle import pack_bits
    return pack_bits(A)


@pytest.mark.parametrize("seed", range(3))
def test_compaction_random_tiny(seed):
    """Tiny random graphs with many labels-alike vertices: compaction after
    every round, hub pieces of 2 entries."""
    from paper_1912_08453_gb300 import ccpm
    ctx = ccpm.Context(0)
    rng = np.random.default_rng(100 + seed)
    n = 60
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.15]
    g = wl.graph_from_edge_list(n, edges, rng.integers(0, 3, size=n))
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    for tl, te in (([0, 1, 2, 0], [(0, 1), (1, 2), (2, 3), (3, 0)]),
                   ([0, 1, 2, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)]),
                   ([0, 0, 1], [(0, 1), (1, 2), (0, 2)])):
        ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
        out = run(ccpm, ctx, graph, tl, te, compact=1, hub_degree=2)
        check(out, ref)
    graph.close()
    ctx.close()


def test_compaction_full_size_rmat22():
    """The scale-22 bench graph with the 4-cycle + triangle template: automatic
    compaction (which fires there) against never compacting -- identical
    outputs and counts; the oracle is too slow for the searches at this size,
    so the two GPU runs are compared with each other and with properties the
    result must have (monotone: omega* within the label-initial state)."""
    from paper_1912_08453_gb300 import ccpm
    ctx = ccpm.Context(0)
    g = wl.rmat_graph(22, labels="degree")
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    tl, te = [5, 12, 11, 11, 5, 7], [(0, 1), (1, 2), (2, 3), (3, 0), (2, 4), (3, 4), (4, 5)]
    a = run(ccpm, ctx, graph, tl, te, compact=0)
    b = run(ccpm, ctx, graph, tl, te, compact=-1)
    assert a["counts"]["lcc_compactions"] > 0 and b["counts"]["lcc_compactions"] == 0
    np.testing.assert_array_equal(a["omega"], b["omega"])
    np.testing.assert_array_equal(a["ebits"], b["ebits"])
    assert a["phases"] == b["phases"]
    for k in ("edges_scanned_lcc", "tokens", "match_embeddings", "count_valid", "active_v", "active_e_dir"):
        assert a["counts"][k] == b["counts"][k], k
    lab_mask = np.zeros(256, dtype=np.uint32)
    for q, L in enumerate(tl):
        lab_mask[L] |= 1 << q
    assert not np.any(a["omega"] & ~lab_mask[g.labels])
    graph.close()
    ctx.close()
