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
