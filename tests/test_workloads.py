"""The seeded input recipe: R-MAT graphs in CSR form (symmetric, simple,
sorted), degree labels as the bit length of the degree, Zipf labels with the
stated skew, connected random templates and edit variants, reproducible from
their seeds."""
import numpy as np

from paper_1912_08453_gb300 import workloads as wl


def _check_csr(g):
    rp, col = g.row_ptr, g.col
    assert rp[0] == 0 and rp[-1] == len(col)
    assert np.all(np.diff(rp) >= 0)
    src = np.repeat(np.arange(g.n), np.diff(rp))
    assert not np.any(src == col), "self loop"
    for v in range(g.n):
        row = col[rp[v]:rp[v + 1]]
        assert np.all(np.diff(row) > 0), "row not strictly increasing (unsorted or duplicate)"
    fwd = set(zip(src.tolist(), col.tolist()))
    assert all((b, a) in fwd for a, b in fwd), "asymmetric"


def test_rmat_csr_is_simple_symmetric_sorted():
    g = wl.rmat_graph(10, labels="degree", seed=3)
    assert g.n == 1 << 10
    _check_csr(g)
    # at most 16 * 2^scale undirected draws, stored in both directions
    assert g.m_dir <= 2 * 16 * (1 << 10)


def test_rmat_is_reproducible_and_seeded():
    a = wl.rmat_graph(9, labels="zipf", seed=5)
    b = wl.rmat_graph(9, labels="zipf", seed=5)
    c = wl.rmat_graph(9, labels="zipf", seed=6)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
    assert np.array_equal(a.labels, b.labels)
    assert not (np.array_equal(a.row_ptr, c.row_ptr) and np.array_equal(a.col, c.col))


def test_rmat_skew_concentrates_degree():
    # Graph 500 parameters give a heavier tail than the uniform (0.25 each) case
    skew = wl.rmat_graph(12, labels="degree", seed=2)
    flat = wl.rmat_graph(12, abcd=(0.25, 0.25, 0.25, 0.25), labels="degree", seed=2)
    assert skew.degrees().max() > 4 * flat.degrees().max()


def test_degree_labels_are_bit_length():
    g = wl.rmat_graph(10, labels="degree", seed=4)
    d = g.degrees()
    expect = np.array([int(x).bit_length() for x in d], dtype=np.uint8)   # ceil(log2(d+1))
    assert np.array_equal(g.labels, expect)


def test_zipf_label_frequencies():
    lab = wl.zipf_labels(200000, n_labels=64, s=1.2, seed=7)
    assert lab.min() >= 0 and lab.max() < 64
    f = np.bincount(lab, minlength=64) / len(lab)
    w = (np.arange(64) + 1.0) ** -1.2
    w /= w.sum()
    assert np.allclose(f[:8], w[:8], atol=0.01)


def test_graph_from_edge_list_matches_csr_rules():
    g = wl.graph_from_edge_list(6, [(0, 1), (1, 2), (2, 0), (2, 0), (3, 3), (4, 5)], [0, 1, 2, 0, 1, 2])
    _check_csr(g)
    assert g.m_dir == 8                 # duplicate and self loop dropped, both directions kept


def test_random_templates_connected_and_variants_bounded():
    pool = [1, 2, 3, 4]
    for seed in range(30):
        t = wl.random_template(seed, 6, 2, pool)
        assert t.n0 == 6 and wl.is_connected(t.n0, t.edges)
        assert all(a != b for a, b in t.edges)
        assert len(set(tuple(sorted(e)) for e in t.edges)) == len(t.edges)
        assert set(t.labels) <= set(pool)
    base = wl.Template([5, 12, 11, 11, 5, 7], [(0, 1), (1, 2), (2, 3), (3, 0), (2, 4), (3, 4), (4, 5)])
    vs = wl.edit_variants(base, 40, seed=5, label_pool=[5, 7, 11, 12])
    assert len(vs) == 40
    assert vs == wl.edit_variants(base, 40, seed=5, label_pool=[5, 7, 11, 12])
    for v in vs:
        assert 5 <= v.n0 <= 9 and wl.is_connected(v.n0, v.edges)


def test_edge_labels_symmetric_seeded_and_weighted():
    g = wl.rmat_graph(10, seed=2)
    el = wl.edge_labels(g.row_ptr, g.col, 4, seed=5)
    assert el.dtype == np.uint8 and el.shape[0] == g.m_dir and el.max() < 4
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    lab = {(int(a), int(b)): int(x) for a, b, x in zip(src, g.col, el)}
    assert all(lab[(b, a)] == x for (a, b), x in lab.items())      # both entries of an edge agree
    assert np.array_equal(el, wl.edge_labels(g.row_ptr, g.col, 4, seed=5))
    assert not np.array_equal(el, wl.edge_labels(g.row_ptr, g.col, 4, seed=6))
    w = wl.edge_labels(g.row_ptr, g.col, 3, seed=5, weights=[8, 1, 1])
    f = np.bincount(w, minlength=3) / len(w)
    assert abs(f[0] - 0.8) < 0.03 and f[1] > 0.05 and f[2] > 0.05


def test_sampled_template_is_a_subgraph_of_the_graph():
    g = wl.rmat_graph(10, seed=3)
    el = wl.edge_labels(g.row_ptr, g.col, 3, seed=1)
    for n0, extra in ((5, 0), (12, 3), (40, 6)):
        tl, te, tel = wl.sampled_template(g, el, n0, extra, seed=n0)
        assert len(tl) == n0 and wl.is_connected(n0, te) and len(te) >= n0 - 1
        assert len(set(te)) == len(te) and all(a < b for a, b in te)
        assert len(tel) == len(te) and set(tl) <= set(int(x) for x in g.labels)
        # the sampled copy itself is a match, so the LCC fixpoint keeps at least n0 vertices
        import oracle
        om, _, _, _ = oracle.wide_lcc(oracle.Graph(g.row_ptr, g.col, g.labels), tl, te, tel, el)
        assert int((om != 0).sum()) >= n0
