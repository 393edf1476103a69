"""Searches that run out of their window budget.

`options.search_budget` bounds the windows one search may scan.  A search that
runs out keeps its root (NLCC, final existence passes) or its edge (final edge
pass), so the result is a superset of the exact answer, the count is reported
invalid and the call returns CCPM_EBUDGET.  With a budget of a few windows
nearly every search runs out; the result must still contain every bit of the
exact result (the oracle's, which has no budget), and the first LCC phase,
which runs before any search, must be identical.
"""
import numpy as np
import pytest

from paper_1912_08453_gb300 import workloads as wl
from oracle import pipeline

pytestmark = pytest.mark.gpu

CYCLE5 = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)]
TL, TE = [0, 1, 2, 0, 0, 5, 0, 0], CYCLE5 + [(2, 5), (5, 6), (3, 7)]
CAP = 1 << 16


@pytest.mark.parametrize("budget", [1, 4, 64])
def test_tiny_budget_gives_a_superset_and_ebudget(budget):
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph(14, labels="zipf")
    ref = pipeline.run(g.row_ptr, g.col, g.labels, TL, TE, max_embeddings=CAP)
    ctx = ccpm.Context(0)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    t = ccpm.Template(ctx, TL, TE)
    h = ccpm.ctypes.c_void_p()
    rc = ccpm.lib.ccpm_prune(ctx.h, graph.h, t.h,
                             ccpm.ctypes.byref(ccpm.options(max_embeddings=CAP, search_budget=budget)),
                             ccpm.ctypes.byref(h))
    assert rc == ccpm.CCPM_EBUDGET, ccpm.lib.ccpm_last_error(ctx.h)
    r = ccpm.Result(graph, h)
    om, eb, c = r.omega(), r.edge_bitmap(), r.counts()
    assert c["status"] == ccpm.CCPM_EBUDGET and c["count_valid"] == 0
    assert not np.any(ref.omega & ~om), "a bit of the exact omega* is missing"
    assert not np.any(ref.ebits & ~eb), "an entry of the exact E* is missing"
    assert r.phase_rounds()[0] == ref.phase_rounds[0]
    # every kept bit is still label-consistent and every kept entry joins live vertices
    assert not np.any(om & ~np.asarray([sum(1 << q for q in range(8) if TL[q] == L) for L in g.labels],
                                       dtype=np.uint32))
    r.close()
    t.close()
    graph.close()
    ctx.close()
