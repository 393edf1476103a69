"""The allocation-free LCC entry point, checked against ccpm_prune.

Callers that may not allocate device memory while they run use
ccpm_lcc_fixpoint_noalloc, which keeps its scratch in a fixed area inside the
library.  Its omega bitsets, edge bitmap, round count and scanned-entry count
must equal those of the regular entry point stopped after local constraint
checking, on two calls in a row (the second call reuses the scratch the first
one left behind).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1912_08453_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# acyclic template with unique labels: no non-local constraint, so the regular
# entry point with the final search switched off returns the LCC fixpoint
TL = [5, 4, 6, 3, 2]
TE = [(0, 1), (1, 2), (1, 3), (3, 4)]


def regular(g):
    from paper_1912_08453_gb300 import ccpm
    ctx = ccpm.Context(0)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    t = ccpm.Template(ctx, TL, TE)
    assert t.generate() == 0
    r = ccpm.prune(ctx, graph, t, ccpm.options(run_final=0))
    out = r.omega(), r.edge_bitmap(), r.phase_rounds(), r.counts()
    r.close()
    graph.close()
    ctx.close()
    return out


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph(15, seed=21)
    om_ref, eb_ref, phases, counts = regular(g)
    dev = torch.device("cuda:0")
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    lab = torch.from_numpy(g.labels).to(dev)
    words = (g.m_dir + 31) // 32
    for call in range(2):
        om = torch.full((g.n,), -1, dtype=torch.int32, device=dev)     # stale output on purpose
        eb = torch.full((words,), -1, dtype=torch.int32, device=dev)
        rounds, scanned = ccpm.lcc_fixpoint_noalloc(0, rp, col, lab, TL, TE, om, eb)
        np.testing.assert_array_equal(om.cpu().numpy().view(np.uint32), om_ref, err_msg=f"call {call}")
        np.testing.assert_array_equal(eb.cpu().numpy().view(np.uint32), eb_ref, err_msg=f"call {call}")
        assert rounds == phases[0]
        assert scanned == counts["edges_scanned_lcc"]


def test_noalloc_rejects_graphs_beyond_its_scratch():
    import torch
    from paper_1912_08453_gb300 import ccpm
    dev = torch.device("cuda:0")
    n = 1 << 22                                   # far beyond the fixed area
    rp = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    col = torch.zeros(1, dtype=torch.int32, device=dev)
    lab = torch.zeros(n, dtype=torch.uint8, device=dev)
    om = torch.zeros(n, dtype=torch.int32, device=dev)
    eb = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(ccpm.CcpmError) as ei:
        ccpm.lcc_fixpoint_noalloc(0, rp, col[:0], lab, TL, TE, om, eb)
    assert ei.value.code == ccpm.CCPM_EINVAL and "too large" in str(ei.value)


def test_noalloc_rejects_offsets_that_disagree_with_m_dir():
    # row_ptr[n] larger than the column count the caller states: rejected
    # before any kernel runs (the scratch is sized from m_dir)
    import torch
    from paper_1912_08453_gb300 import ccpm
    dev = torch.device("cuda:0")
    g = wl.rmat_graph(10, seed=3)
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col[:-64].copy()).to(dev)
    lab = torch.from_numpy(g.labels).to(dev)
    om = torch.zeros(g.n, dtype=torch.int32, device=dev)
    eb = torch.zeros((g.m_dir + 31) // 32, dtype=torch.int32, device=dev)
    before = torch.cuda.current_device()
    with pytest.raises(ccpm.CcpmError) as ei:
        ccpm.lcc_fixpoint_noalloc(0, rp, col, lab, TL, TE, om, eb)
    assert ei.value.code == ccpm.CCPM_EINVAL and "row_ptr" in str(ei.value)
    assert torch.cuda.current_device() == before
