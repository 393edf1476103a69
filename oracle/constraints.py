"""Non-local constraint generation for the oracle (TEST INFRASTRUCTURE).

Plain Python restatement of the paper's Table 3 procedure (Steps 1-5) and of
Alg. 2 (TDS_CONSTRAINTS), with the ordering heuristic of Section 4.2
("Constraint Ordering Heuristics").  Shares no code with the product's C++
constraint generator; the tests compare the two lists element by element.

Readings taken where the paper is silent (each is listed with its reason in the
design notes):
  * FIND_CIRCLES returns every simple cycle (length >= 3) of G'_0, one per edge
    set, in lexicographic order of the canonical vertex sequence (start at the
    smallest id, second vertex smaller than the last).
  * FIND_SHORTEST_PATH(G0, qi, qj, 3) returns the lexicographically smallest
    shortest qi -> qj path when dist(qi, qj) >= 3, else nothing.  A path whose
    edges all lie on one cycle constraint is dropped (Step 4, optimisation ii).
  * Alg. 2 merges pairs repeatedly, always the first mergeable pair (i, j) in
    index order, until no pair merges.  Cycle lists merge on a shared vertex
    plus a shared edge; path lists and the Step 5(3) mixed list merge on a
    shared vertex alone.  Path-derived results are replaced by the BFS spanning
    tree from their lowest-id vertex (neighbours in increasing id); the mixed
    list keeps all its edges.
  * K0 = PC + CC + TDS_CC + TDS_PC + TDS with exact duplicates (same vertex and
    edge set) removed, first occurrence kept; then stably ordered by
    (is TDS, number of edges, kind rank PC < CC < TDS_CC < TDS_PC < TDS,
    generation index).
  * Heads (Section 4.2 "Token Generation"): every vertex of a cycle or of a
    cycle-derived TDS; both terminals of a path; for path-derived and mixed TDS
    the vertices of S whose label repeats in the template (all of S if none).
"""
from __future__ import annotations

from collections import deque

KIND_PC, KIND_CC, KIND_TDS_CC, KIND_TDS_PC, KIND_TDS = 0, 1, 2, 3, 4
KIND_NAMES = {KIND_PC: "PC", KIND_CC: "CC", KIND_TDS_CC: "TDS_CC",
              KIND_TDS_PC: "TDS_PC", KIND_TDS: "TDS"}
MAX_CYCLES = 4096


class Constraint:
    def __init__(self, kind, verts, edges):
        self.kind = kind
        self.verts = frozenset(verts)
        self.edges = frozenset(tuple(sorted(e)) for e in edges)
        self.heads = frozenset()

    def key(self):
        return (self.verts, self.edges)

    def vmask(self):
        m = 0
        for v in self.verts:
            m |= 1 << v
        return m

    def hmask(self):
        m = 0
        for v in self.heads:
            m |= 1 << v
        return m

    def sadj(self, n0):
        """Adjacency within S as template-id bitmasks."""
        out = [0] * 32
        for a, b in self.edges:
            out[a] |= 1 << b
            out[b] |= 1 << a
        return out

    def __repr__(self):
        return f"{KIND_NAMES[self.kind]}(V={sorted(self.verts)}, E={sorted(self.edges)}, H={sorted(self.heads)})"


def _adjacency(n0, edges):
    adj = [set() for _ in range(n0)]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    return adj


def find_cycles(verts, edges):
    """All simple cycles of the graph (verts, edges), each once."""
    vs = sorted(verts)
    adj = {v: set() for v in vs}
    for a, b in edges:
        if a in adj and b in adj:
            adj[a].add(b)
            adj[b].add(a)
    out = []

    def dfs(start, path, onpath):
        x = path[-1]
        for y in sorted(adj[x]):
            if y == start and len(path) >= 3 and path[1] < path[-1]:
                out.append(list(path))
                if len(out) > MAX_CYCLES:
                    raise ValueError("template has too many simple cycles")
            elif y > start and y not in onpath:
                path.append(y)
                onpath.add(y)
                dfs(start, path, onpath)
                onpath.discard(y)
                path.pop()

    for s in vs:
        dfs(s, [s], {s})
    out.sort()
    return out


def shortest_path_lex(adj, src, dst):
    """Lexicographically smallest shortest path src -> dst (None if unreachable)."""
    dist = {dst: 0}
    q = deque([dst])
    while q:
        x = q.popleft()
        for y in adj[x]:
            if y not in dist:
                dist[y] = dist[x] + 1
                q.append(y)
    if src not in dist:
        return None
    path = [src]
    x = src
    while x != dst:
        x = min(y for y in adj[x] if dist.get(y, -1) == dist[x] - 1)
        path.append(x)
    return path


def bfs_spanning_tree(verts, edges):
    vs = sorted(verts)
    adj = {v: set() for v in vs}
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    root = vs[0]
    seen = {root}
    q = deque([root])
    tree = []
    while q:
        x = q.popleft()
        for y in sorted(adj[x]):
            if y not in seen:
                seen.add(y)
                tree.append((min(x, y), max(x, y)))
                q.append(y)
    return tree


def tds_constraints(items, mode):
    """Alg. 2.  mode: 'CC' (needs a shared edge), 'PC' or 'MIX' (shared vertex)."""
    work = [(set(c.verts), set(c.edges)) for c in items]
    while True:
        merged = False
        for i in range(len(work)):
            for j in range(i + 1, len(work)):
                vi, ei = work[i]
                vj, ej = work[j]
                if not (vi & vj):
                    continue
                if mode == "CC" and not (ei & ej):
                    continue
                work[i] = (vi | vj, ei | ej)
                del work[j]
                merged = True
                break
            if merged:
                break
        if not merged:
            break
    if mode == "PC":
        work = [(v, set(bfs_spanning_tree(v, e))) for v, e in work]
    return work


def generate(labels, edges):
    """Ordered non-local constraint set K0 for template (labels, edges)."""
    n0 = len(labels)
    adj = _adjacency(n0, edges)
    count = {}
    for L in labels:
        count[L] = count.get(L, 0) + 1
    # Step 1: unique-label leaves are left to LCC
    v_u = {q for q in range(n0) if count[labels[q]] == 1}
    v_ul = {q for q in v_u if len(adj[q]) == 1}
    v1 = set(range(n0)) - v_ul
    e1 = [(a, b) for a, b in edges if a in v1 and b in v1]
    # Step 2: duplicate-label vertices
    v_d = set(range(n0)) - v_u
    # Step 3: cycle constraints
    cc = []
    for cyc in find_cycles(v1, e1):
        ed = [(cyc[i], cyc[(i + 1) % len(cyc)]) for i in range(len(cyc))]
        cc.append(Constraint(KIND_CC, cyc, ed))
    # Step 4: path constraints between same-label pairs three or more hops apart
    pc = []
    for i in sorted(v_d):
        for j in sorted(v_d):
            if j <= i or labels[i] != labels[j]:
                continue
            path = shortest_path_lex(adj, i, j)
            if path is None or len(path) - 1 < 3:
                continue
            ed = [(path[k], path[k + 1]) for k in range(len(path) - 1)]
            c = Constraint(KIND_PC, path, ed)
            if any(c.edges <= x.edges for x in cc):
                continue
            pc.append(c)
    # Step 5: TDS constraints
    tds_cc = [Constraint(KIND_TDS_CC, v, e) for v, e in tds_constraints(cc, "CC")]
    tds_pc = [Constraint(KIND_TDS_PC, v, e) for v, e in tds_constraints(pc, "PC")]
    tds = [Constraint(KIND_TDS, v, e) for v, e in tds_constraints(tds_cc + tds_pc, "MIX")]
    k0 = []
    seen = set()
    for c in pc + cc + tds_cc + tds_pc + tds:
        if c.key() in seen:
            continue
        seen.add(c.key())
        k0.append(c)
    for c in k0:
        if c.kind in (KIND_CC, KIND_TDS_CC):
            c.heads = c.verts
        elif c.kind == KIND_PC:
            c.heads = frozenset(q for q in c.verts if len([e for e in c.edges if q in e]) == 1)
        else:
            dup = c.verts & v_d
            c.heads = dup if dup else c.verts
    order = sorted(range(len(k0)),
                   key=lambda i: (1 if k0[i].kind >= KIND_TDS_CC else 0,
                                  len(k0[i].edges), k0[i].kind, i))
    return [k0[i] for i in order]
