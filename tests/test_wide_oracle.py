"""Pins of the oracle's LCC for wider templates (up to 64 vertices, 64-bit
omega) and edge labels (Section 5.1's eight-byte omega; Section 3's edge
metadata), independent of the oracle itself:

* with every edge label 0 and at most 32 template vertices it is the 32-bit
  LCC of the pinned oracle (same omega, edge flags, rounds, scanned entries);
* every match survives (brute force with edge labels, tiny graphs), and for
  acyclic templates with unique vertex labels nothing else does;
* planted 40- and 64-vertex paths: exactly the correct copy survives;
* hand-derived cases: an edge label that breaks a triangle (round count by
  hand), the multiplicity rule counted per edge label, and coverage checked
  per template neighbour where the multiplicity of its class is met;
* monotone rounds that reach a fixpoint.
"""
import numpy as np
import pytest

import oracle
from paper_1912_08453_gb300 import workloads as wl
from tests.bruteforce import truth_labelled


def graph_of(n, edges, labels, elabel=None):
    """CSR of an undirected edge list; elabel: {(a, b): label} (symmetric)."""
    g = wl.graph_from_edge_list(n, edges, labels)
    el = None
    if elabel is not None:
        el = np.zeros(g.m_dir, dtype=np.uint8)
        for v in range(n):
            for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
                u = int(g.col[e])
                el[e] = elabel[(min(v, u), max(v, u))]
    return g, el


def random_graph(rng, n, p, n_labels, n_elabels):
    edges, elabel = [], {}
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < p:
                edges.append((a, b))
                elabel[(a, b)] = int(rng.integers(0, n_elabels))
    labels = rng.integers(0, n_labels, size=n)
    return graph_of(n, edges, labels, elabel)


def random_tree(rng, n0, labels, n_elabels):
    edges = [(int(rng.integers(0, v)), v) for v in range(1, n0)]
    tel = [int(rng.integers(0, n_elabels)) for _ in edges]
    return list(labels), edges, tel


@pytest.mark.parametrize("seed", range(6))
def test_reduces_to_the_32_bit_lcc_without_edge_labels(seed):
    g = wl.rmat_graph(9, seed=seed + 1)
    pool = [L for L in wl.labels_by_frequency(g) if L > 0][:5]
    t = wl.random_template(seed, 4 + seed % 5, seed % 3, pool)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A = oracle.init(og, t.labels, t.edges)
    rounds, scanned = oracle.lcc(og, t.labels, t.edges, om, A)
    for el, tel in ((None, None), (np.zeros(g.m_dir, dtype=np.uint8), [0] * len(t.edges))):
        om64, A64, r64, s64 = oracle.wide_lcc(og, t.labels, t.edges, tel, el)
        np.testing.assert_array_equal(om64, om.astype(np.uint64))
        np.testing.assert_array_equal(A64, A)
        assert (r64, s64) == (rounds, scanned)


@pytest.mark.parametrize("seed", range(12))
def test_every_match_survives_with_edge_labels(seed):
    rng = np.random.default_rng(100 + seed)
    g, el = random_graph(rng, 11, 0.45, 3, 2)
    n0 = 3 + seed % 3
    labels = [int(x) for x in rng.integers(0, 3, size=n0)]
    tl, te, tel = random_tree(rng, n0, labels, 2)
    if seed % 2:                      # close a cycle
        te = te + [(0, n0 - 1)] if (0, n0 - 1) not in te else te
        tel = tel + [int(rng.integers(0, 2))] if len(tel) < len(te) else tel
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A, _, _ = oracle.wide_lcc(og, tl, te, tel, el)
    om_t, A_t, count = truth_labelled(g.row_ptr, g.col, g.labels, tl, te, tel, el)
    assert not np.any(om_t & ~om), "a vertex of a match was pruned"
    assert not np.any(A_t & (1 - A)), "an edge of a match was pruned"


@pytest.mark.parametrize("seed", range(10))
def test_exact_for_trees_with_unique_vertex_labels(seed):
    rng = np.random.default_rng(200 + seed)
    n0 = 3 + seed % 4
    tl, te, tel = random_tree(rng, n0, range(n0), 3)
    g, el = random_graph(rng, 40, 0.12, n0, 3)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A, _, _ = oracle.wide_lcc(og, tl, te, tel, el)
    om_t, A_t, count = truth_labelled(g.row_ptr, g.col, g.labels, tl, te, tel, el)
    np.testing.assert_array_equal(om, om_t)
    np.testing.assert_array_equal(A, A_t)


def planted_paths(n0, rng):
    """Three copies of an n0-vertex path labelled 0..n0-1 with edge labels
    1, 2, 1, 2, ...: copy 0 intact, copy 1 with one middle edge relabelled,
    copy 2 missing its middle edge; plus noise edges (labels 1..2) that join
    copies at random."""
    edges, elabel = [], {}
    labels = []
    for c in range(3):
        base = c * n0
        labels += list(range(n0))
        for i in range(n0 - 1):
            if c == 2 and i == n0 // 2:
                continue
            L = 1 + i % 2
            if c == 1 and i == n0 // 2:
                L = 3 - L
            edges.append((base + i, base + i + 1))
            elabel[(base + i, base + i + 1)] = L
    n = 3 * n0
    while len(edges) < 3 * (n0 - 1) + n0:
        a, b = sorted(int(x) for x in rng.integers(0, n, size=2))
        if a != b and (a, b) not in elabel:
            edges.append((a, b))
            elabel[(a, b)] = int(rng.integers(1, 3))
    return graph_of(n, edges, labels, elabel)


@pytest.mark.parametrize("n0", [40, 64])
def test_planted_long_path_is_found_exactly(n0):
    rng = np.random.default_rng(n0)
    g, el = planted_paths(n0, rng)
    tl = list(range(n0))
    te = [(i, i + 1) for i in range(n0 - 1)]
    tel = [1 + i % 2 for i in range(n0 - 1)]
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A, rounds, _ = oracle.wide_lcc(og, tl, te, tel, el)
    om_t, A_t, count = truth_labelled(g.row_ptr, g.col, g.labels, tl, te, tel, el)
    assert count >= 1
    np.testing.assert_array_equal(om, om_t)
    np.testing.assert_array_equal(A, A_t)
    # the intact copy keeps every template vertex, the top bit included
    assert all(int(om[v]) == 1 << v for v in range(n0))
    assert int(om[n0 - 1]) >> (n0 - 1) == 1


def test_edge_label_breaks_a_triangle():
    # template triangle q0-q1-q2 (labels 0, 1, 2), every edge labelled 1;
    # graph triangle with the same vertex labels, edge (0, 2) labelled 2
    tl, te, tel = [0, 1, 2], [(0, 1), (1, 2), (0, 2)], [1, 1, 1]
    g, el = graph_of(3, [(0, 1), (1, 2), (0, 2)], [0, 1, 2], {(0, 1): 1, (1, 2): 1, (0, 2): 2})
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A, rounds, _ = oracle.wide_lcc(og, tl, te, tel, el)
    # first LCC round: entries (0,2) and (2,0) fail eta, so vertices 0 and 2
    # lose the only neighbour that could cover them; second: vertex 1 has no
    # live neighbour left; the third changes nothing
    assert not om.any() and not A.any()
    assert rounds == 3
    # the same graph with every edge labelled 1 matches
    el1 = np.ones_like(el)
    om, A, rounds, _ = oracle.wide_lcc(og, tl, te, tel, el1)
    assert [int(x) for x in om] == [1, 2, 4] and A.all() and rounds == 1


def test_multiplicity_is_counted_per_edge_label():
    # template star: centre q0 (label 0) with leaves q1, q2 (label 5) joined
    # by edge label 1 and q3 (label 5) joined by edge label 2
    tl, te, tel = [0, 5, 5, 5], [(0, 1), (0, 2), (0, 3)], [1, 1, 2]
    # centres 0 and 8 match (two label-5 leaves by label 1, one by label 2);
    # centre 4 has three label-5 leaves but only one by edge label 1, while
    # its leaf 6 (joined by label 2) can be a label-1 leaf of centre 8
    edges = [(0, 1), (0, 2), (0, 3), (4, 5), (4, 6), (4, 7), (8, 6), (8, 9), (8, 10)]
    elabel = {(0, 1): 1, (0, 2): 1, (0, 3): 2, (4, 5): 1, (4, 6): 2, (4, 7): 2,
              (6, 8): 1, (8, 9): 1, (8, 10): 2}
    g, el = graph_of(11, edges, [0, 5, 5, 5, 0, 5, 5, 5, 0, 5, 5], elabel)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A, _, _ = oracle.wide_lcc(og, tl, te, tel, el)
    om_t, A_t, count = truth_labelled(g.row_ptr, g.col, g.labels, tl, te, tel, el)
    np.testing.assert_array_equal(om, om_t)
    np.testing.assert_array_equal(A, A_t)
    assert int(om[0]) == 1 and int(om[8]) == 1 and int(om[4]) == 0 and count == 4
    # without edge labels centre 4 would pass the count of label-5 leaves
    om0, _, _, _ = oracle.wide_lcc(og, tl, te, None, None)
    assert int(om0[4]) == 1


def test_coverage_is_checked_per_template_neighbour():
    # template path a - b - c plus a - d: a and c share label 0 (b: 1, d: 3),
    # every edge labelled 1.  Vertex 0 (label 1) has two label-0 neighbours,
    # neither with a label-3 neighbour, so both can only be c: two
    # neighbours meet {a, c} (the multiplicity of the class) but none holds a.
    # By hand: vertices 1, 2 and 5 lose a (no label-3 neighbour), so vertex 0
    # sees c twice but never a and dies, and then 1 and 2 lose c; vertex 3
    # keeps b (4 holds a and c, 5 holds c), 4 keeps {a, c}, 6 keeps d.  (c in
    # omega(4) is a false positive only a non-local check removes.)
    tl, te, tel = [0, 1, 0, 3], [(0, 1), (1, 2), (0, 3)], [1, 1, 1]
    edges = [(0, 1), (0, 2), (3, 4), (3, 5), (4, 6)]
    g, el = graph_of(7, edges, [1, 0, 0, 1, 0, 0, 3], {e: 1 for e in edges})
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A, _, _ = oracle.wide_lcc(og, tl, te, tel, el)
    assert [int(x) for x in om] == [0, 0, 0, 0b10, 0b101, 0b100, 0b1000]
    om_t, A_t, count = truth_labelled(g.row_ptr, g.col, g.labels, tl, te, tel, el)
    assert count == 1 and not np.any(om_t & ~om) and not np.any(A_t & (1 - A))


def test_rounds_are_monotone_and_reach_a_fixpoint():
    g = wl.rmat_graph(8, seed=4)
    el = wl.edge_labels(g.row_ptr, g.col, 3, seed=9)
    pool = [L for L in wl.labels_by_frequency(g) if L > 0][:4]
    t = wl.random_template(5, 6, 2, pool)
    tel = [i % 3 for i in range(len(t.edges))]
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A = oracle.wide_init(og, t.labels)
    k = 0
    while True:
        ch, om2, A2, _ = oracle.wide_lcc_round(og, t.labels, t.edges, om, A, tel, el)
        k += 1
        assert not np.any(om2 & ~om) and not np.any(A2 & (1 - A))
        om, A = om2, A2
        if not ch:
            break
    om_f, A_f, rounds, _ = oracle.wide_lcc(og, t.labels, t.edges, tel, el)
    assert rounds == k
    np.testing.assert_array_equal(om, om_f)
    np.testing.assert_array_equal(A, A_f)
    ch, om3, A3, _ = oracle.wide_lcc_round(og, t.labels, t.edges, om, A, tel, el)
    assert not ch and np.array_equal(om3, om) and np.array_equal(A3, A)
