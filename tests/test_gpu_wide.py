"""GPU LCC for templates of up to 64 vertices with edge labels
(ccpm_lcc_wide) vs the oracle, through the C ABI, bit-exact: 64-bit omega
words, edge-bitmap words, rounds, active entries scanned, and the active
vertex / entry totals."""
import numpy as np
import pytest

import oracle
from paper_1912_08453_gb300 import workloads as wl
from tests.test_wide_oracle import planted_paths

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1912_08453_gb300 import ccpm
    return ccpm.Context(0)


def check(ctx, g, tl, te, tel=None, el=None, el_on_device=False):
    from paper_1912_08453_gb300 import ccpm
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    keep = None
    if el is not None:
        if el_on_device:
            import torch
            keep = torch.from_numpy(el).cuda()
            graph.set_edge_labels(keep)
        else:
            graph.set_edge_labels(el, validate=True)
    om, bits, st = ccpm.lcc_wide(ctx, graph, tl, te, tel)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om_r, A_r, rounds, scanned = oracle.wide_lcc(og, tl, te, tel, el)
    np.testing.assert_array_equal(om, om_r)
    np.testing.assert_array_equal(bits, oracle.pack_bits(A_r))
    assert st["rounds"] == rounds and st["edges_scanned"] == scanned
    assert st["active_v"] == int((om_r != 0).sum()) and st["active_e_dir"] == int(A_r.sum())
    graph.close()
    del keep
    return om, st


def test_equals_the_first_fixpoint_of_prune(ctx):
    # no edge labels, 32-bit template: the first LCC fixpoint of ccpm_prune
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph(14, seed=5)
    tl, te = [5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)]
    om, st = check(ctx, g, tl, te)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    t = ccpm.Template(ctx, tl, te)
    r = ccpm.prune(ctx, graph, t, ccpm.options(lcc_only=1))
    np.testing.assert_array_equal(om, r.omega().astype(np.uint64))
    assert r.phase_rounds()[0] == st["rounds"]
    r.close()


@pytest.mark.parametrize("n0,extra,scale,n_el", [(6, 1, 14, 2), (12, 3, 14, 3), (33, 4, 16, 2),
                                                  (48, 6, 16, 3), (64, 8, 16, 2), (64, 0, 14, 1)])
def test_sampled_templates_with_edge_labels(ctx, n0, extra, scale, n_el):
    g = wl.rmat_graph(scale, seed=n0 + scale)
    el = wl.edge_labels(g.row_ptr, g.col, n_el, seed=n0, weights=[8] + [1] * (n_el - 1))
    tl, te, tel = wl.sampled_template(g, el, n0, extra, seed=n0)
    om, st = check(ctx, g, tl, te, tel, el)
    assert st["active_v"] >= n0          # the sampled copy itself survives


@pytest.mark.parametrize("n0", [40, 64])
def test_planted_long_paths(ctx, n0):
    g, el = planted_paths(n0, np.random.default_rng(n0))
    tl = list(range(n0))
    te = [(i, i + 1) for i in range(n0 - 1)]
    tel = [1 + i % 2 for i in range(n0 - 1)]
    om, st = check(ctx, g, tl, te, tel, el)
    assert [int(x) for x in om[:n0]] == [1 << v for v in range(n0)]


def test_device_edge_labels_and_ragged_rows(ctx):
    # borrowed device labels; a zipf-labelled graph whose rows straddle
    # bitmap words at every offset
    g = wl.rmat_graph(13, seed=9, labels="zipf")
    el = wl.edge_labels(g.row_ptr, g.col, 4, seed=2)
    tl, te, tel = wl.sampled_template(g, el, 20, 5, seed=3)
    check(ctx, g, tl, te, tel, el, el_on_device=True)


def test_device_outputs(ctx):
    # outputs written to device memory hold the same words as host outputs
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph(12, seed=4)
    el = wl.edge_labels(g.row_ptr, g.col, 2, seed=1)
    tl, te, tel = wl.sampled_template(g, el, 36, 3, seed=7)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    graph.set_edge_labels(el)
    om_h, bits_h, st_h = ccpm.lcc_wide(ctx, graph, tl, te, tel)
    om_d, bits_d, st_d = ccpm.lcc_wide(ctx, graph, tl, te, tel, device_out=True)
    np.testing.assert_array_equal(om_d.cpu().numpy().view(np.uint64), om_h)
    np.testing.assert_array_equal(bits_d.cpu().numpy().view(np.uint32), bits_h)
    assert st_d["rounds"] == st_h["rounds"] and st_d["edges_scanned"] == st_h["edges_scanned"]
    graph.close()


def test_nothing_active(ctx):
    # template labels absent from the graph: one quiescent round, empty result
    g = wl.rmat_graph(10, seed=2)
    tl, te = [250, 251, 252], [(0, 1), (1, 2)]
    om, st = check(ctx, g, tl, te)
    assert st["rounds"] == 1 and not om.any()


def test_template_checks(ctx):
    from paper_1912_08453_gb300 import ccpm
    g = wl.rmat_graph(8, seed=1)
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    path65 = [(i, i + 1) for i in range(64)]
    for tl, te, tel, msg in (([0] * 65, path65, None, "2..64 vertices"),
                             ([0, 1, 2, 3], [(0, 1), (2, 3)], None, "not connected"),
                             ([0] * 10, [(i, i + 1) for i in range(9)], list(range(9)), "more than 8 edge labels"),
                             ([0, 1], [(0, 1), (1, 0)], None, "duplicate")):
        with pytest.raises(ccpm.CcpmError, match=msg):
            ccpm.lcc_wide(ctx, graph, tl, te, tel)
    bad = np.zeros(graph.m, dtype=np.uint8)
    bad[0] = 1                            # one direction of an edge only
    with pytest.raises(ccpm.CcpmError, match="differ"):
        graph.set_edge_labels(bad, validate=True)
