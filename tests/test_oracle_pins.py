"""Pins for the CPU oracle: checks against things other than the oracle itself.

* brute-force enumeration of every injective labelled map on tiny graphs
  (Definition 1): the pruned output equals the union of all matches, and
  before the final search it is a superset (100% recall);
* invariants: pruning is monotone, the LCC result is a fixpoint, and a
  Gauss-Seidel schedule reaches the same fixpoint;
* acyclic unique-label templates: LCC alone is exact (Section 4);
* the Fig. 2(a) and Fig. 2(c) constructions;
* closed-form counts on unlabelled graphs (traces of adjacency powers);
* hand-derived constraint sets (Table 3, Alg. 2);
* order invariance of the final result.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import constraints as cgen
from oracle import pipeline
from paper_1912_08453_gb300 import workloads as wl
from bruteforce import truth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_graph(seed, n, p, n_labels):
    rng = np.random.default_rng(seed)
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < p]
    labels = rng.integers(0, n_labels, size=n)
    return wl.graph_from_edge_list(n, edges, labels)


TEMPLATES = [
    ("triangle", [0, 1, 2], [(0, 1), (1, 2), (0, 2)]),
    ("triangle-rep", [0, 0, 1], [(0, 1), (1, 2), (0, 2)]),
    ("path4-rep", [0, 1, 2, 0], [(0, 1), (1, 2), (2, 3)]),
    ("c4", [0, 1, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 0)]),
    ("star3", [0, 1, 1, 1], [(0, 1), (0, 2), (0, 3)]),
    ("k4", [0, 1, 2, 0], [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
    ("k5-e", [0, 1, 2, 0, 1], [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3), (0, 4), (1, 4), (2, 4)]),
    ("tree-tri", [1, 0, 2, 1, 0], [(0, 1), (1, 2), (1, 3), (2, 3), (3, 4)]),
    ("c5", [0, 1, 2, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)]),
    ("path5-rep", [2, 0, 1, 0, 2], [(0, 1), (1, 2), (2, 3), (3, 4)]),
]


def bit_subset(a, b):
    """a is a subset of b element-wise (uint arrays)."""
    return bool(np.all((a & ~b) == 0))


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("tname,tl,te", TEMPLATES, ids=[t[0] for t in TEMPLATES])
def test_bruteforce_exact(seed, tname, tl, te):
    n_labels = max(tl) + 1
    g = random_graph(1000 + seed, 9, 0.45, n_labels)
    wt, At, cnt = truth(g.row_ptr, g.col, g.labels, tl, te)
    r = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    assert r.count_valid
    assert r.match_embeddings == cnt
    np.testing.assert_array_equal(r.omega, wt)
    np.testing.assert_array_equal(r.A, At)
    # recall: the state before the final search already contains every match
    assert bit_subset(wt, r.omega_pre_final)
    assert bit_subset(At, r.A_pre_final)
    # M_sub counts distinct subgraphs: each one is found |Aut| times
    assert r.match_embeddings % r.automorphisms == 0


def test_bruteforce_denser_graphs():
    for seed in range(4):
        g = random_graph(77 + seed, 10, 0.6, 2)
        for tl, te in [([0, 1, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 0)]),
                       ([0, 0, 0], [(0, 1), (1, 2), (0, 2)]),
                       ([0, 1, 1, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0), (0, 2)])]:
            wt, At, cnt = truth(g.row_ptr, g.col, g.labels, tl, te)
            r = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
            assert r.match_embeddings == cnt
            np.testing.assert_array_equal(r.omega, wt)
            np.testing.assert_array_equal(r.A, At)


@pytest.mark.parametrize("seed", range(4))
def test_monotone_and_fixpoint(seed):
    g = random_graph(200 + seed, 30, 0.2, 3)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    tl, te = [0, 1, 2, 0], [(0, 1), (1, 2), (2, 3), (3, 0), (0, 2)]
    om, A = oracle.init(og, tl, te)
    rounds = 0
    while True:
        ch, om2, A2, _ = oracle.lcc_round(og, tl, te, om, A)
        rounds += 1
        assert bit_subset(om2, om), "omega gained a template vertex"
        assert np.all(A2 <= A), "an eliminated edge came back"
        changed_truly = bool(np.any(om2 != om) or np.any(A2 != A))
        assert ch == changed_truly
        om, A = om2, A2
        if not ch:
            break
    # a further round changes nothing (fixpoint), and the loop counted it
    ch, om3, A3, _ = oracle.lcc_round(og, tl, te, om, A)
    assert not ch
    om_b, A_b = oracle.init(og, tl, te)
    r, _ = oracle.lcc(og, tl, te, om_b, A_b)
    assert r == rounds
    np.testing.assert_array_equal(om_b, om)
    # NLCC is monotone too
    for c in cgen.generate(tl, te):
        before_om, before_A = om.copy(), A.copy()
        oracle.nlcc(og, c.vmask(), c.sadj(len(tl)), c.hmask(), om, A)
        assert bit_subset(om, before_om)
        assert np.all(A <= before_A)


def gauss_seidel_lcc(g, tl, te, order_seed):
    """LCC with in-place updates in a random vertex order (test-only schedule)."""
    n = g.n
    n0 = len(tl)
    adj = [0] * n0
    for a, b in te:
        adj[a] |= 1 << b
        adj[b] |= 1 << a
    om = [0] * n
    for v in range(n):
        for q in range(n0):
            if tl[q] == g.labels[v]:
                om[v] |= 1 << q
    nbrs = [[int(u) for u in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]] for v in range(n)]
    act = {(v, u): bool(om[v] and om[u]) for v in range(n) for u in nbrs[v]}

    def compat(x, y):
        return any((x >> a) & 1 and adj[a] & y for a in range(n0))

    rng = np.random.default_rng(order_seed)
    changed = True
    while changed:
        changed = False
        for v in rng.permutation(n):
            v = int(v)
            if not om[v]:
                continue
            live = []
            for u in nbrs[v]:
                if act[(v, u)] and compat(om[v], om[u]):
                    live.append(u)
                elif act[(v, u)]:
                    act[(v, u)] = act[(u, v)] = False
                    changed = True
            union = 0
            for u in live:
                union |= om[u]
            keep = 0
            for q in range(n0):
                if not (om[v] >> q) & 1 or (adj[q] & ~union):
                    continue
                ok = True
                for L in set(tl[b] for b in range(n0) if (adj[q] >> b) & 1):
                    group = sum(1 << b for b in range(n0) if (adj[q] >> b) & 1 and tl[b] == L)
                    if sum(1 for u in live if om[u] & group) < bin(group).count("1"):
                        ok = False
                if ok:
                    keep |= 1 << q
            if not live:
                keep = 0
            if keep != om[v]:
                om[v] = keep
                changed = True
            if not keep:
                for u in nbrs[v]:
                    if act[(v, u)]:
                        act[(v, u)] = act[(u, v)] = False
                        changed = True
    A = np.array([1 if act[(v, int(g.col[e]))] else 0
                  for v in range(n) for e in range(g.row_ptr[v], g.row_ptr[v + 1])], dtype=np.uint8)
    return np.array(om, dtype=np.uint32), A


@pytest.mark.parametrize("seed", range(4))
def test_schedule_independence(seed):
    g = random_graph(300 + seed, 40, 0.12, 3)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    tl, te = [0, 1, 2, 1], [(0, 1), (1, 2), (2, 3), (1, 3)]
    om, A = oracle.init(og, tl, te)
    oracle.lcc(og, tl, te, om, A)
    for s in range(3):
        om_gs, A_gs = gauss_seidel_lcc(g, tl, te, s)
        np.testing.assert_array_equal(om, om_gs)
        np.testing.assert_array_equal(A, A_gs)


def test_acyclic_unique_labels_lcc_exact():
    # Section 4: LCC alone is precise for acyclic templates with unique labels.
    tl, te = [0, 1, 2, 3, 4], [(0, 1), (1, 2), (1, 3), (3, 4)]
    assert cgen.generate(tl, te) == []
    for seed in range(5):
        g = random_graph(400 + seed, 9, 0.4, 5)
        wt, At, cnt = truth(g.row_ptr, g.col, g.labels, tl, te)
        og = oracle.Graph(g.row_ptr, g.col, g.labels)
        om, A = oracle.init(og, tl, te)
        oracle.lcc(og, tl, te, om, A)
        np.testing.assert_array_equal(om, wt)
        np.testing.assert_array_equal(A, At)


def _fixture_graph(fx):
    gd = fx["graph"]
    return wl.graph_from_edge_list(gd["n"], gd["edges"], gd["labels"])


def test_fig2a_cycle_needs_cycle_check():
    fx = json.load(open(os.path.join(GOLDEN, "fig2a_cycle9.json")))
    g = _fixture_graph(fx)
    tl = fx["template"]["labels"]
    te = [tuple(e) for e in fx["template"]["edges"]]
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A = oracle.init(og, tl, te)
    oracle.lcc(og, tl, te, om, A)
    assert int(np.count_nonzero(om)) == fx["expect"]["survive_lcc"]
    assert int(np.count_nonzero(A)) == fx["expect"]["survive_lcc_edges_dir"]
    K = cgen.generate(tl, te)
    assert [(cgen.KIND_NAMES[c.kind], sorted(c.verts), sorted(c.heads)) for c in K] == \
        [(c["kind"], c["verts"], c["heads"]) for c in fx["expect"]["constraints"]]
    oracle.nlcc(og, K[0].vmask(), K[0].sadj(3), K[0].hmask(), om, A)
    assert int(np.count_nonzero(om)) == fx["expect"]["after_cc"]
    r = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    assert r.match_embeddings == fx["expect"]["matches"]


def test_fig2c_torus_needs_tds():
    fx = json.load(open(os.path.join(GOLDEN, "fig2c_torus.json")))
    g = _fixture_graph(fx)
    tl = fx["template"]["labels"]
    te = [tuple(e) for e in fx["template"]["edges"]]
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A = oracle.init(og, tl, te)
    oracle.lcc(og, tl, te, om, A)
    K = cgen.generate(tl, te)
    for c in K:
        if c.kind == cgen.KIND_CC:
            ch, _ = oracle.nlcc(og, c.vmask(), c.sadj(5), c.hmask(), om, A)
            if ch:
                oracle.lcc(og, tl, te, om, A)
    assert int(np.count_nonzero(om)) == fx["expect"]["survive_lcc_and_cycles"]
    for c in K:
        if c.kind != cgen.KIND_CC:
            ch, _ = oracle.nlcc(og, c.vmask(), c.sadj(5), c.hmask(), om, A)
            if ch:
                oracle.lcc(og, tl, te, om, A)
    assert int(np.count_nonzero(om)) == fx["expect"]["after_tds"]
    wt, _, cnt = truth(g.row_ptr, g.col, g.labels, tl, te)
    assert cnt == fx["expect"]["matches"] and not wt.any()


def _adj_matrix(g):
    n = g.n
    M = np.zeros((n, n), dtype=np.int64)
    for v in range(n):
        M[v, g.col[g.row_ptr[v]:g.row_ptr[v + 1]]] = 1
    return M


@pytest.mark.parametrize("scale", [7, 8])
def test_unlabelled_closed_forms(scale):
    g = wl.rmat_graph(scale, seed=scale)
    g.labels = np.zeros(g.n, dtype=np.uint8)
    M = _adj_matrix(g)
    d = M.sum(1)
    cases = [
        ([0, 0, 0], [(0, 1), (1, 2), (0, 2)], int(np.trace(M @ M @ M))),
        ([0, 0, 0], [(0, 1), (1, 2)], int(np.sum(d * (d - 1)))),
        ([0, 0, 0, 0], [(0, 1), (0, 2), (0, 3)], int(np.sum(d * (d - 1) * (d - 2)))),
        ([0, 0, 0, 0], [(0, 1), (1, 2), (2, 3), (3, 0)],
         int(np.trace(M @ M @ M @ M) - 2 * np.sum(d * d) + np.sum(d))),
    ]
    for tl, te, expect in cases:
        r = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
        assert r.count_valid
        assert r.match_embeddings == expect, (te, r.match_embeddings, expect)


def test_constraint_generation_hand_derived():
    fx = json.load(open(os.path.join(GOLDEN, "constraint_generation.json")))
    for case in fx["cases"]:
        K = cgen.generate(case["labels"], [tuple(e) for e in case["edges"]])
        got = [{"kind": cgen.KIND_NAMES[c.kind], "verts": sorted(c.verts),
                "edges": sorted([list(e) for e in c.edges]), "heads": sorted(c.heads)} for c in K]
        assert got == case["expect"], case["name"]


@pytest.mark.parametrize("seed", range(3))
def test_order_invariance(seed):
    g = random_graph(500 + seed, 10, 0.5, 2)
    tl, te = [0, 1, 0, 1, 0], [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (1, 4)]
    K = cgen.generate(tl, te)
    assert len(K) >= 3
    base = pipeline.run(g.row_ptr, g.col, g.labels, tl, te, constraints=K)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        perm = [K[i] for i in rng.permutation(len(K))]
        r = pipeline.run(g.row_ptr, g.col, g.labels, tl, te, constraints=perm)
        np.testing.assert_array_equal(r.omega, base.omega)
        np.testing.assert_array_equal(r.A, base.A)
        assert r.match_embeddings == base.match_embeddings


def test_budget_reports_invalid_count_but_exact_sets():
    # past the cap the count is invalid; omega* and E* are still exact
    for seed in range(4):
        g = random_graph(800 + seed, 9, 0.5, 2)
        for tl, te in [([0, 1, 0], [(0, 1), (1, 2)]), ([0, 1, 0, 1], [(0, 1), (1, 2), (2, 3), (3, 0)])]:
            wt, At, cnt = truth(g.row_ptr, g.col, g.labels, tl, te)
            if cnt < 3:
                continue
            r = pipeline.run(g.row_ptr, g.col, g.labels, tl, te, max_embeddings=1)
            assert not r.count_valid and r.match_embeddings == 0
            np.testing.assert_array_equal(r.omega, wt)
            np.testing.assert_array_equal(r.A, At)


@pytest.mark.parametrize("k", [2, 3])
def test_star_multiplicity_lcc_exact(k):
    # A star whose k leaves share one label: a centre needs k distinct active
    # neighbours with that label (the multiplicity rule of Section 4.1 / Section 4.3).
    # For stars that rule makes LCC exact, so it is pinned by brute force.
    tl = [0] + [1] * k
    te = [(0, i) for i in range(1, k + 1)]
    for seed in range(6):
        g = random_graph(600 + seed, 10, 0.3, 2)
        wt, At, cnt = truth(g.row_ptr, g.col, g.labels, tl, te)
        og = oracle.Graph(g.row_ptr, g.col, g.labels)
        om, A = oracle.init(og, tl, te)
        oracle.lcc(og, tl, te, om, A)
        np.testing.assert_array_equal(om, wt)
        np.testing.assert_array_equal(A, At)


def _nlcc_by_definition(g, omega, A, S_verts, S_edges, heads):
    """Alg. 6 from its definition, by trying every injective map of S."""
    import itertools
    n = g.n
    entry = {}
    for v in range(n):
        for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
            entry[(v, int(g.col[e]))] = e
    S = sorted(S_verts)
    om = omega.copy()
    for h in sorted(heads):
        for v in range(n):
            if not (int(omega[v]) >> h) & 1:
                continue
            sat = False
            for img in itertools.permutations(range(n), len(S)):
                psi = dict(zip(S, img))
                if psi[h] != v:
                    continue
                if any(not (int(omega[psi[q]]) >> q) & 1 for q in S):
                    continue
                if all((psi[a], psi[b]) in entry and A[entry[(psi[a], psi[b])]] for a, b in S_edges):
                    sat = True
                    break
            if not sat:
                om[v] &= ~np.uint32(1 << h)
    A2 = A.copy()
    for v in range(n):
        for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
            u = int(g.col[e])
            if (omega[v] and not om[v]) or (omega[u] and not om[u]):
                A2[e] = 0
    return om, A2


@pytest.mark.parametrize("seed", range(12))
def test_nlcc_against_definition(seed):
    # Arbitrary snapshots (not only LCC fixpoints): random omega subsets of the
    # label-compatible sets, random symmetric edge flags with dead endpoints off,
    # so that edges with live endpoints but no active flag occur.
    rng = np.random.default_rng(seed)
    tl = [0, 1, 0, 1, 2]
    te = [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (2, 4)]
    g = random_graph(700 + seed, 8, 0.7, 3)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om0, A0 = oracle.init(og, tl, te)
    keep = np.zeros(g.n, dtype=np.uint32)
    for q in range(len(tl)):
        keep |= (rng.random(g.n) < 0.85).astype(np.uint32) << np.uint32(q)
    om0 = om0 & keep
    A0 = A0.copy()
    for v in range(g.n):
        for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
            u = int(g.col[e])
            if u > v and rng.random() < 0.3:
                A0[e] = 0
                A0[g.row_ptr[u] + np.searchsorted(g.col[g.row_ptr[u]:g.row_ptr[u + 1]], v)] = 0
            if not om0[v] or not om0[u]:
                A0[e] = 0
    for c in cgen.generate(tl, te):
        om, A = om0.copy(), A0.copy()
        oracle.nlcc(og, c.vmask(), c.sadj(len(tl)), c.hmask(), om, A)
        om_d, A_d = _nlcc_by_definition(g, om0, A0, c.verts, c.edges, c.heads)
        np.testing.assert_array_equal(om, om_d, err_msg=str(c))
        np.testing.assert_array_equal(A, A_d, err_msg=str(c))


def test_scanned_counts_active_entries():
    # The edges-scanned metric: the entries read by a round are the active
    # entries of active vertices at the start of that round.
    g = random_graph(901, 40, 0.2, 3)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    tl, te = [0, 1, 2], [(0, 1), (1, 2)]
    om, A = oracle.init(og, tl, te)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    expect = int(np.sum(A[(om[src] != 0)]))
    _, _, _, sc = oracle.lcc_round(og, tl, te, om, A)
    assert sc == expect


def _compat_state(g, tl, te, om):
    """[both ends live and compat(omega(v), omega(u))] per CSR entry (eta of
    Alg. 4, written out from the template's adjacency)."""
    adj = [0] * len(tl)
    for a, b in te:
        adj[a] |= 1 << b
        adj[b] |= 1 << a
    nbr = np.zeros(len(om), dtype=np.uint64)
    for q in range(len(tl)):
        nbr |= np.where((om.astype(np.uint64) >> np.uint64(q)) & np.uint64(1), np.uint64(adj[q]), np.uint64(0))
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    omu = om.astype(np.uint64)
    return ((omu[src] != 0) & (omu[g.col] != 0) & ((nbr[src] & omu[g.col]) != 0)).astype(np.uint8)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("tname,tl,te", TEMPLATES[:8], ids=[t[0] for t in TEMPLATES[:8]])
def test_fixpoint_edges_are_compat_on_live_pairs(seed, tname, tl, te):
    """At every LCC fixpoint (after the first LCC and after each non-local
    constraint's re-run) an entry is active exactly when both ends are live
    and their omegas are compatible: bits are cleared only by a failed eta or
    a dead end, and eta stays true once omega only shrinks.  The searches
    rely on this instead of reading the edge flags."""
    g = random_graph(900 + seed, 32, 0.25, max(tl) + 1)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A = oracle.init(og, tl, te)
    oracle.lcc(og, tl, te, om, A)
    np.testing.assert_array_equal(A, _compat_state(g, tl, te, om))
    for c in cgen.generate(tl, te):
        ch, _ = oracle.nlcc(og, c.vmask(), c.sadj(len(tl)), c.hmask(), om, A)
        if ch:
            oracle.lcc(og, tl, te, om, A)
        np.testing.assert_array_equal(A, _compat_state(g, tl, te, om))


def _tree_diameter(n0, edges):
    adj = [[] for _ in range(n0)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    best = 0
    for s in range(n0):
        dist = {s: 0}
        frontier = [s]
        while frontier:
            nxt = []
            for x in frontier:
                for y in adj[x]:
                    if y not in dist:
                        dist[y] = dist[x] + 1
                        nxt.append(y)
            frontier = nxt
        best = max(best, max(dist.values()))
    return best


@pytest.mark.parametrize("seed", range(40))
def test_lcc_rounds_within_diameter_bound(seed):
    """Acyclic templates with unique labels: LCC settles within diam(G0) + 1
    rounds (Sec. 5.1's k_max), counting the final round that changes
    nothing.  (Exactness of LCC for this class is pinned separately.)"""
    rng = np.random.default_rng(4000 + seed)
    n0 = int(rng.integers(2, 8))
    te = [(int(rng.integers(0, v)), v) for v in range(1, n0)]
    tl = [int(x) for x in rng.permutation(n0)]
    n = int(rng.integers(15, 40))
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < float(rng.uniform(0.08, 0.3))]
    g = wl.graph_from_edge_list(n, edges, rng.integers(0, n0, size=n))
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    om, A = oracle.init(og, tl, te)
    rounds, _ = oracle.lcc(og, tl, te, om, A)
    assert rounds <= _tree_diameter(n0, te) + 1


@pytest.mark.parametrize("L", range(1, 14))
def test_jacobi_rounds_peel_a_path_one_layer_per_round(L):
    """Exact round count of snapshot (Jacobi) rounds, computed by hand.

    Triangle template, all labels 0: a template vertex needs two distinct live
    neighbours.  On a path of L vertices (all label 0) only the two ends lack
    them; in a snapshot round a vertex sees its neighbours as they were at the
    start of the round, so round k removes exactly the vertices k-1 steps from
    an end.  The path is empty after ceil(L/2) rounds and one more round
    changes nothing: ceil(L/2) + 1 rounds in all.  An in-place (Gauss-Seidel)
    sweep in index order would empty it in its first round (2 rounds)."""
    g = wl.graph_from_edge_list(L, [(i, i + 1) for i in range(L - 1)], [0] * L)
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    tl, te = [0, 0, 0], [(0, 1), (1, 2), (0, 2)]
    om, A = oracle.init(og, tl, te)
    # round by round: the set removed in round k is {k-1, L-k}
    alive = set(range(L))
    for k in range(1, (L + 1) // 2 + 1):
        ch, om, A, _ = oracle.lcc_round(og, tl, te, om, A)
        assert ch
        alive -= {k - 1, L - k}
        assert set(np.flatnonzero(om).tolist()) == alive, f"round {k}"
    om, A = oracle.init(og, tl, te)
    rounds, _ = oracle.lcc(og, tl, te, om, A)
    assert rounds == (L + 1) // 2 + 1
    assert not om.any() and not A.any()


def test_edge_only_change_counts_a_round():
    """A round that removes an entry but no omega bit still counts as a
    change (Alg. 4 sets the change flag for eliminated edges): 2 rounds.

    Template q0 (label 0) - q1 (label 1).  Background: a (0) - b (1) and
    a (0) - c (0).  First LCC round: the entry a-c is not compatible (no template
    edge joins q0 to q0) and is removed; a keeps q0 through b, b keeps q1,
    c has no compatible neighbour and dies.  The second round changes nothing."""
    g = wl.graph_from_edge_list(3, [(0, 1), (0, 2)], [0, 1, 0])
    og = oracle.Graph(g.row_ptr, g.col, g.labels)
    tl, te = [0, 1], [(0, 1)]
    om, A = oracle.init(og, tl, te)
    rounds, _ = oracle.lcc(og, tl, te, om, A)
    assert rounds == 2
    assert om.tolist() == [1, 2, 0]
    # entries of row 0 are (0,1), (0,2); row 1: (1,0); row 2: (2,0)
    assert A.tolist() == [1, 0, 1, 0]
    # and with c given label 1 instead, nothing is removed: one quiet round
    g2 = wl.graph_from_edge_list(3, [(0, 1), (0, 2)], [0, 1, 1])
    og2 = oracle.Graph(g2.row_ptr, g2.col, g2.labels)
    om, A = oracle.init(og2, tl, te)
    rounds, _ = oracle.lcc(og2, tl, te, om, A)
    assert rounds == 1 and A.all()


def test_openmp_build_gives_identical_results():
    """The OpenMP build of the oracle parallelises only loops whose
    iterations write disjoint words (or set flags to 1): every output equals
    the single-threaded build's, including the existence passes past the
    count cap."""
    g = wl.rmat_graph(12, labels="zipf", seed=9)
    cyc = [(0, 1), (1, 2), (2, 3), (3, 4), (4, 0)]
    tl, te = [0, 1, 2, 0, 0, 5, 0, 0], cyc + [(2, 5), (5, 6), (3, 7)]
    runs = []
    for par in (False, True):
        oracle.set_parallel(par)
        try:
            runs.append(pipeline.run(g.row_ptr, g.col, g.labels, tl, te, max_embeddings=1 << 10))
        finally:
            oracle.set_parallel(False)
    a, b = runs
    assert not a.count_valid            # the existence passes ran
    np.testing.assert_array_equal(a.omega, b.omega)
    np.testing.assert_array_equal(a.A, b.A)
    np.testing.assert_array_equal(a.omega_pre_final, b.omega_pre_final)
    assert a.phase_rounds == b.phase_rounds and a.lcc_scanned == b.lcc_scanned
    assert a.tokens == b.tokens
    # (entries scanned by the edge pass are not compared: an entry another
    # thread has already marked is skipped, so that metric depends on timing)
