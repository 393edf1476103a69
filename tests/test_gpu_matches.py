"""Match listing and participation counts on the GPU (ccpm_result_matches)
against brute force on tiny graphs and against the oracle's listing at the
scale-16 workload: the same set of matches, the same per-vertex and
per-entry counts, bit for bit."""
import numpy as np
import pytest

import oracle
from oracle import pipeline
from paper_1912_08453_gb300 import workloads as wl
from test_oracle_matches import TEMPLATES, brute, random_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1912_08453_gb300 import ccpm
    return ccpm.Context(0)


def gpu_matches(ctx, g, tl, te, list_cap, device=False, **opt):
    from paper_1912_08453_gb300 import ccpm
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    t = ccpm.Template(ctx, tl, te)
    r = ccpm.prune(ctx, graph, t, ccpm.options(**opt), allow_budget=True)
    out = r.matches(t, list_cap=list_cap, vertex_counts=True, entry_counts=True, device=device)
    if device:
        out = (out[0], out[1].cpu().numpy(), out[2].cpu().numpy().astype(np.uint64),
               out[3].cpu().numpy().astype(np.uint64))
    r.close()
    t.close()
    graph.close()
    return out


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("ti", range(len(TEMPLATES)))
def test_tiny_listing_equals_brute_force(ctx, seed, ti):
    tl, te = TEMPLATES[ti]
    g = random_graph(700 + seed, 12, 0.35, max(tl) + 1)
    phis, vc_t, ec_t = brute(g, tl, te)
    for device in (False, True):
        cnt, lst, vc, ec = gpu_matches(ctx, g, tl, te, 10 ** 5, device=device)
        assert cnt == len(phis)
        assert sorted(map(tuple, lst.tolist())) == sorted(phis)
        np.testing.assert_array_equal(vc, vc_t)
        np.testing.assert_array_equal(ec, ec_t)


def test_rmat16_listing_equals_oracle(ctx):
    g = wl.rmat_graph(16)
    tl, te = [5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)]
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    cnt_o, lst_o, vc_o, ec_o = oracle.matches(og, tl, te, ref.omega, ref.A, list_cap=10 ** 6)
    assert cnt_o == ref.match_embeddings > 0
    cnt, lst, vc, ec = gpu_matches(ctx, g, tl, te, 10 ** 6)
    assert cnt == cnt_o
    np.testing.assert_array_equal(np.unique(lst, axis=0), np.unique(lst_o, axis=0))
    assert len(np.unique(lst, axis=0)) == cnt
    np.testing.assert_array_equal(vc, vc_o)
    np.testing.assert_array_equal(ec, ec_o)
    # a listing cap below the count: every count stays exact, the rows are
    # distinct matches
    cnt2, lst2, vc2, ec2 = gpu_matches(ctx, g, tl, te, 100)
    assert cnt2 == cnt and lst2.shape == (100, 6)
    assert len(np.unique(lst2, axis=0)) == 100
    assert set(map(tuple, lst2.tolist())) <= set(map(tuple, lst_o.tolist()))
    np.testing.assert_array_equal(vc2, vc_o)
    np.testing.assert_array_equal(ec2, ec_o)
