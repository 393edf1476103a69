"""Exhaustive labelled subgraph-monomorphism enumeration for tiny graphs.

Independent of the oracle: it tries every injective map of the template's
vertices into the graph (Definition 1 of the paper: labels preserved, every
template edge mapped onto a graph edge) and reports the union of all matches.
"""
import itertools

import numpy as np


def enumerate_matches(n, edge_set, labels, tlabels, tedges):
    n0 = len(tlabels)
    for phi in itertools.permutations(range(n), n0):
        if any(labels[phi[q]] != tlabels[q] for q in range(n0)):
            continue
        if all((phi[a], phi[b]) in edge_set for a, b in tedges):
            yield phi


def truth(row_ptr, col, labels, tlabels, tedges):
    """(omega*, A*, count): per-vertex template sets, per-entry flags, #matches."""
    n = len(row_ptr) - 1
    edge_set = set()
    index = {}
    for v in range(n):
        for e in range(row_ptr[v], row_ptr[v + 1]):
            edge_set.add((v, int(col[e])))
            index[(v, int(col[e]))] = e
    omega = np.zeros(n, dtype=np.uint32)
    A = np.zeros(len(col), dtype=np.uint8)
    count = 0
    for phi in enumerate_matches(n, edge_set, labels, tlabels, tedges):
        count += 1
        for q, v in enumerate(phi):
            omega[v] |= np.uint32(1 << q)
        for a, b in tedges:
            A[index[(phi[a], phi[b])]] = 1
            A[index[(phi[b], phi[a])]] = 1
    return omega, A, count


def truth_labelled(row_ptr, col, labels, tlabels, tedges, tedge_labels=None, edge_labels=None):
    """(omega* as uint64 [n], A* uint8 [m], count) with edge labels, for
    templates of up to 64 vertices.

    Every injective map that preserves vertex labels and maps each template
    edge onto a graph edge of the same label is enumerated by backtracking
    over the template vertices in breadth-first order: a partial map is only
    extended by vertices that already satisfy the constraints to the placed
    vertices, which skips no complete match (independent of the oracle)."""
    n = len(row_ptr) - 1
    n0 = len(tlabels)
    tel = list(tedge_labels) if tedge_labels is not None else [0] * len(tedges)
    elab = {}
    index = {}
    nbrs = [[] for _ in range(n)]
    for v in range(n):
        for e in range(row_ptr[v], row_ptr[v + 1]):
            u = int(col[e])
            elab[(v, u)] = int(edge_labels[e]) if edge_labels is not None else 0
            index[(v, u)] = e
            nbrs[v].append(u)
    tadj = [dict() for _ in range(n0)]
    for (a, b), L in zip(tedges, tel):
        tadj[a][b] = L
        tadj[b][a] = L
    order = [0]
    seen = {0}
    for q in order:
        for b in sorted(tadj[q]):
            if b not in seen:
                seen.add(b)
                order.append(b)
    assert len(order) == n0, "template must be connected"
    pos = {q: i for i, q in enumerate(order)}
    phi = [-1] * n0
    used = set()
    omega = [0] * n
    A = np.zeros(len(col), dtype=np.uint8)
    count = 0

    def fits(q, v):
        if labels[v] != tlabels[q] or v in used:
            return False
        for b, L in tadj[q].items():
            if pos[b] < pos[q] and elab.get((phi[b], v)) != L:
                return False
        return True

    def rec(i):
        nonlocal count
        if i == n0:
            count += 1
            for q in range(n0):
                omega[phi[q]] |= 1 << q
            for (a, b) in tedges:
                A[index[(phi[a], phi[b])]] = 1
                A[index[(phi[b], phi[a])]] = 1
            return
        q = order[i]
        placed = [b for b in tadj[q] if pos[b] < i]
        cands = range(n) if not placed else nbrs[phi[placed[0]]]
        for v in cands:
            if fits(q, v):
                phi[q] = v
                used.add(v)
                rec(i + 1)
                used.discard(v)
                phi[q] = -1

    rec(0)
    return np.array(omega, dtype=np.uint64), A, count
