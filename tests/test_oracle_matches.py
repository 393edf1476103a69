"""The oracle's match listing and participation counts, pinned by brute force.

Every injective label-preserving map that sends template edges onto graph
edges (Definition 1) is enumerated by tests/bruteforce.py.  The oracle's
listing must hold exactly those maps (as a set), and its per-vertex and
per-entry counts must equal the number of brute-force matches that contain the
vertex / map a template edge onto the entry's edge -- whether it enumerates
inside the exact pruned state or inside the initial (unpruned) one."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import pipeline
from paper_1912_08453_gb300 import workloads as wl
from bruteforce import enumerate_matches

TEMPLATES = [
    ([0, 1, 2], [(0, 1), (1, 2), (0, 2)]),
    ([0, 0, 1], [(0, 1), (1, 2), (0, 2)]),
    ([0, 1, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 0)]),
    ([0, 1, 1, 1], [(0, 1), (0, 2), (0, 3)]),
    ([2, 0, 1, 0, 2], [(0, 1), (1, 2), (2, 3), (3, 4)]),
]


def random_graph(seed, n, p, n_labels):
    rng = np.random.default_rng(seed)
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
    return wl.graph_from_edge_list(n, edges, rng.integers(0, n_labels, size=n))


def brute(g, tl, te):
    edge_set, index = set(), {}
    for v in range(g.n):
        for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
            edge_set.add((v, int(g.col[e])))
            index[(v, int(g.col[e]))] = e
    phis = list(enumerate_matches(g.n, edge_set, g.labels, tl, te))
    vc = np.zeros(g.n, dtype=np.uint64)
    ec = np.zeros(g.m_dir, dtype=np.uint64)
    for phi in phis:
        for v in phi:
            vc[v] += 1
        for a, b in te:
            ec[index[(phi[a], phi[b])]] += 1
            ec[index[(phi[b], phi[a])]] += 1
    return phis, vc, ec


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("ti", range(len(TEMPLATES)))
def test_listing_and_counts_equal_brute_force(seed, ti):
    tl, te = TEMPLATES[ti]
    g = random_graph(700 + seed, 12, 0.35, max(tl) + 1)
    phis, vc_t, ec_t = brute(g, tl, te)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    r = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    om0, A0 = oracle.init(og, tl, te)
    for om, A in ((r.omega, r.A), (om0, A0)):
        cnt, lst, vc, ec = oracle.matches(og, tl, te, om, A, list_cap=10 ** 6)
        assert cnt == len(phis)
        assert sorted(map(tuple, lst.tolist())) == sorted(phis)
        np.testing.assert_array_equal(vc, vc_t)
        np.testing.assert_array_equal(ec, ec_t)


def test_listing_stops_at_its_cap_but_counts_everything():
    tl, te = [0, 0, 0], [(0, 1), (1, 2), (0, 2)]
    # K5, all labels 0: 5*4*3 = 60 triangle embeddings.  A vertex is in
    # 3 positions x 4*3 images of the other two = 36 of them; an edge {x, y}
    # is the image of 3 template edges x 2 orientations x 3 choices of the
    # third vertex = 18 of them.
    g = wl.graph_from_edge_list(5, list(itertools.combinations(range(5), 2)), [0] * 5)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A = oracle.init(og, tl, te)
    cnt, lst, vc, ec = oracle.matches(og, tl, te, om, A, list_cap=7)
    assert cnt == 60 and lst.shape == (7, 3)
    assert set(map(tuple, lst.tolist())) <= set(itertools.permutations(range(5), 3))
    assert vc.tolist() == [36] * 5
    assert ec.tolist() == [18] * 20
