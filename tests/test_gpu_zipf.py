"""Skewed labels with repeated template labels and a 5-cycle: the template
class that needs the template-driven search (TDS) constraints of Table 3.

R-MAT scale 14 with Zipf(1.2) labels over 64 labels (iid per vertex), the
small stand-in of the scale-25 configuration.  With labels independent of
the structure these templates have millions of matches, so the final count is
capped: both sides must then report the count invalid and still return the
exact omega* and E* (existence searches past the cap).  Parity is bit-exact
on omega, the edge bitmap, LCC rounds per phase, tokens and active entries
scanned; the compaction modes must not change any of it.
"""
import numpy as np
import pytest

from paper_1912_08453_gb300 import workloads as wl
from oracle import pipeline
from oracle import constraints as cgen

pytestmark = pytest.mark.gpu

CYCLE5 = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)]
TEMPLATES = [
    ([0, 1, 2, 0, 0, 5, 0, 0], CYCLE5 + [(2, 5), (5, 6), (3, 7)]),
    ([0, 5, 5, 1, 1, 1, 3, 0], CYCLE5 + [(2, 5), (5, 6), (3, 7)]),
    ([2, 1, 3, 1, 5, 0, 2, 1], CYCLE5 + [(2, 5), (5, 6), (3, 7)]),
    ([0, 0, 1, 1, 4, 2, 1, 0], CYCLE5 + [(1, 5), (5, 6), (6, 7), (7, 3)]),
]
CAP = 1 << 16


@pytest.fixture(scope="module")
def env():
    from paper_1912_08453_gb300 import ccpm
    ctx = ccpm.Context(0)
    g = wl.rmat_graph(14, labels="zipf")
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    yield ccpm, ctx, g, graph
    graph.close()
    ctx.close()


@pytest.mark.parametrize("ti", range(len(TEMPLATES)))
def test_zipf_tds_parity(env, ti):
    ccpm, ctx, g, graph = env
    tl, te = TEMPLATES[ti]
    kinds = {c.kind for c in cgen.generate(tl, te)}
    assert kinds & {2, 3, 4}, "template must produce TDS constraints"
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te, max_embeddings=CAP)
    for mode in (0, 1, -1):
        t = ccpm.Template(ctx, tl, te)
        r = ccpm.prune(ctx, graph, t, ccpm.options(max_embeddings=CAP, compact=mode), allow_budget=True)
        c = r.counts()
        np.testing.assert_array_equal(r.omega(), ref.omega)
        np.testing.assert_array_equal(r.edge_bitmap(), ref.ebits)
        assert r.phase_rounds() == ref.phase_rounds
        assert c["count_valid"] == int(ref.count_valid)
        assert c["match_embeddings"] == ref.match_embeddings
        assert c["tokens"] == ref.tokens
        assert c["edges_scanned_lcc"] == ref.lcc_scanned
        r.close()
        t.close()
