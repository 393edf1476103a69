"""Long searches hand their untried candidates on as new items, run in further
passes.  With search_split = 1 every search splits after its first window, so
nearly all search work goes through that path: results must stay bit-exact
against the oracle (omega, edge bitmap, rounds per phase, tokens, counts),
for the non-local constraints, the final count and marking, and past the
count cap."""
import numpy as np
import pytest

from paper_1912_08453_gb300 import workloads as wl
from oracle import pipeline

pytestmark = pytest.mark.gpu

TEMPLATES = [
    ([0, 1, 2], [(0, 1), (1, 2), (0, 2)]),
    ([0, 1, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 0)]),
    ([0, 1, 2, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)]),
    ([0, 1, 2, 0], [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
    ([0, 0, 1, 1, 2], [(0, 1), (1, 2), (2, 3), (3, 0), (2, 4), (3, 4)]),
]


def run(ctx, g, tl, te, **opt):
    from paper_1912_08453_gb300 import ccpm
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    t = ccpm.Template(ctx, tl, te)
    r = ccpm.prune(ctx, graph, t, ccpm.options(**opt), allow_budget=True)
    out = dict(omega=r.omega(), ebits=r.edge_bitmap(), counts=r.counts(), phases=r.phase_rounds())
    r.close(); t.close(); graph.close()
    return out


def check(out, ref):
    np.testing.assert_array_equal(out["omega"], ref.omega)
    np.testing.assert_array_equal(out["ebits"], ref.ebits)
    assert out["phases"] == ref.phase_rounds
    assert out["counts"]["tokens"] == ref.tokens
    assert out["counts"]["match_embeddings"] == ref.match_embeddings
    assert out["counts"]["count_valid"] == int(ref.count_valid)


@pytest.fixture(scope="module")
def ctx():
    from paper_1912_08453_gb300 import ccpm
    return ccpm.Context(0)


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("ti", range(len(TEMPLATES)))
def test_split_every_search_tiny(ctx, seed, ti):
    rng = np.random.default_rng(700 + seed)
    n = 40
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.25]
    tl, te = TEMPLATES[ti]
    g = wl.graph_from_edge_list(n, edges, rng.integers(0, max(tl) + 1, size=n))
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    for mode in (1, -1):
        check(run(ctx, g, tl, te, search_split=1, compact=mode), ref)


@pytest.mark.parametrize("cap", [1 << 32, 1 << 10])
def test_split_every_search_rmat16(ctx, cap):
    g = wl.rmat_graph(16, labels="degree")
    tl, te = [7, 8, 7, 4, 4, 6], [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 5)]
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te, max_embeddings=cap)
    for split in (1, 7, -1):
        check(run(ctx, g, tl, te, search_split=split, max_embeddings=cap), ref)


def test_split_zipf_tds(ctx):
    g = wl.rmat_graph(14, labels="zipf")
    tl = [0, 1, 2, 0, 0, 5, 0, 0]
    te = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (2, 5), (5, 6), (3, 7)]
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te, max_embeddings=1 << 16)
    for split in (1, 64):
        check(run(ctx, g, tl, te, search_split=split, max_embeddings=1 << 16), ref)
