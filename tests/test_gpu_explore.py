"""Exploratory search (ccpm_explore) against independent prunes and the oracle.

The driver relaxes an over-constrained base template level by level (k edges
removed, connected variants only) and stops at the first level where some
variant has a match.  Each variant is pruned from the candidate set (the
union of every variant's LCC fixpoint) instead of from the label-initial
state; its omega*, E* and count must equal a prune of that variant alone, the
level found must be the first level at which independent prunes find a match,
and the union returned must be the union of those variants' omega* and E*."""
import numpy as np
import pytest

from oracle import pipeline
from paper_1912_08453_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def variants_at(base_l, base_e, k):
    import itertools
    out = []
    for rem in itertools.combinations(range(len(base_e)), k):
        ed = [e for i, e in enumerate(base_e) if i not in rem]
        if ed and wl.is_connected(len(base_l), ed):
            out.append((sum(1 << i for i in rem), ed))
    return out


@pytest.mark.parametrize("base_l,base_e,max_k", [
    # a 5-clique: no match until four edges are removed (the first matches at
    # level 4; one at level 2 for the second label set)
    ([5, 6, 5, 6, 7], [(0, 1), (0, 2), (0, 3), (0, 4), (1, 2), (1, 3), (1, 4), (2, 3), (2, 4), (3, 4)], 4),
    ([6, 7, 6, 7, 8], [(0, 1), (0, 2), (0, 3), (0, 4), (1, 2), (1, 3), (1, 4), (2, 3), (2, 4), (3, 4)], 3),
    # a 4-cycle plus a chord and a tail
    ([5, 6, 5, 6, 7], [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2), (3, 4)], 2),
])
def test_explore_equals_independent_prunes(base_l, base_e, max_k):
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph(13, labels="degree", seed=17)
    ctx = ccpm.Context(0)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    base = ccpm.Template(ctx, base_l, base_e)
    level, union, recs, ms_c = ccpm.explore(ctx, graph, base, max_k)
    # independent prunes, level by level
    expect_level, om_u, eb_u = -1, np.zeros(g.n, np.uint32), np.zeros(graph.words, np.uint32)
    by_mask = {}
    for k in range(max_k + 1):
        any_match = False
        for mask, ed in variants_at(base_l, base_e, k):
            t = ccpm.Template(ctx, base_l, ed)
            r = ccpm.prune(ctx, graph, t)
            om, eb, c = r.omega(), r.edge_bitmap(), r.counts()
            by_mask[mask] = (om, eb, c)
            if c["active_v"] > 0:
                any_match = True
                om_u |= om
                eb_u |= eb
            r.close()
            t.close()
        if any_match:
            expect_level = k
            break
    assert level == expect_level
    assert len(recs) == len(by_mask)
    for rec in recs:
        om, eb, c = by_mask[rec["removed"]]
        assert rec["active_v"] == c["active_v"] and rec["active_e_dir"] == c["active_e_dir"]
        assert rec["match_embeddings"] == c["match_embeddings"]
    np.testing.assert_array_equal(union.omega(), om_u)
    np.testing.assert_array_equal(union.edge_bitmap(), eb_u)
    # the first matching variant also equals the oracle
    if level >= 0:
        rec = next(r for r in recs if r["level"] == level and r["active_v"] > 0)
        ed = [e for i, e in enumerate(base_e) if not (rec["removed"] >> i) & 1]
        ref = pipeline.run(g.row_ptr, g.col, g.labels, base_l, ed)
        np.testing.assert_array_equal(by_mask[rec["removed"]][0], ref.omega)
    union.close()
    graph.close()
    ctx.close()
