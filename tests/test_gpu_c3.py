"""C3 at its stated size, and its whole pipeline one scale down.

C3 is R-MAT scale 25 (edge factor 16: about 1.05e9 CSR entries once
symmetrised), Zipf(1.2) labels over 64 labels, and an 8-vertex template with
repeated labels and a 5-cycle, whose non-local constraints include
template-driven searches.

* Scale 25: the first LCC fixpoint (omega words, edge-bitmap words, rounds,
  active entries scanned) equals the oracle's (its OpenMP build), bit for
  bit.  The template shape is taken over the most frequent labels: about
  half the vertices start active and omega (134 MB) no longer fits in L2.
  The launch configuration is the one the benchmark times (options.lcc_only).
* Scale 20: the whole pipeline of the C3 template as benchmarked (labels from
  the Zipf tail) equals the oracle's: omega*, E*, rounds per phase, tokens,
  and the count (capped: invalid on both sides).
"""
import numpy as np
import pytest

import bench
import oracle
from oracle import pipeline
from paper_1912_08453_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_scale25_first_lcc_fixpoint_equals_oracle():
    import torch
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph_philox(25, labels="zipf", device="cuda:0")
    torch.cuda.synchronize()
    assert g.n == 1 << 25 and g.m_dir > 10 ** 9
    ctx = ccpm.Context(0)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    tl, te = bench.C3_FREQUENT
    t = ccpm.Template(ctx, tl, te)
    r = ccpm.prune(ctx, graph, t, ccpm.options(lcc_only=1))
    om, eb, c, ph = r.omega(), r.edge_bitmap(), r.counts(), r.phase_rounds()
    r.close()
    t.close()
    graph.close()
    h = g.to_host()
    del g
    torch.cuda.empty_cache()
    og = oracle.Graph(h.row_ptr, h.col, h.labels)
    oracle.set_parallel(True)
    try:
        om_o, A_o = oracle.init(og, tl, te)
        rounds, scanned = oracle.lcc(og, tl, te, om_o, A_o)
    finally:
        oracle.set_parallel(False)
    assert ph == [rounds]
    assert c["edges_scanned_lcc"] == scanned
    assert int(np.count_nonzero(om_o)) > 10 ** 6          # a large live set
    np.testing.assert_array_equal(om, om_o)
    # the edge bitmap handed back at an LCC fixpoint (no final search): a bit
    # is set iff the oracle's entry is active
    np.testing.assert_array_equal(eb, oracle.pack_bits(A_o))


def test_scale20_whole_pipeline_equals_oracle():
    import torch
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph_philox(20, labels="zipf", device="cuda:0").to_host()
    torch.cuda.empty_cache()
    tl, te = bench.C3_TEMPLATE
    cap = 1 << 16
    ctx = ccpm.Context(0)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    t = ccpm.Template(ctx, tl, te)
    assert any(d["kind"].startswith("TDS") for d in t.constraints())
    r = ccpm.prune(ctx, graph, t, ccpm.options(max_embeddings=cap), allow_budget=True)
    oracle.set_parallel(True)
    try:
        ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te, max_embeddings=cap)
    finally:
        oracle.set_parallel(False)
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
    graph.close()
