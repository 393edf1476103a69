"""Seeded synthetic inputs: R-MAT background graphs, vertex labels and templates.

This module only *generates inputs*; it holds none of the pruning arithmetic, so
both the CUDA path and the CPU oracle consume its arrays unchanged.

Background graphs follow the R-MAT recipe the paper uses for its synthetic runs
(Section 6 "Datasets", and Section 6.10 for the three (A, B, C, D) skews):
2^scale vertices, edge factor 16 directed draws, undirected by storing both
directions, with self loops and duplicate edges removed.  Vertex labels are
either degree-derived, l(v) = ceil(log2(d(v)+1)) (Section 6 "Datasets"), which
is the bit length of d(v), or Zipf-distributed over a fixed label alphabet.

Randomness: numpy's Philox counter-based bit generator, seeded explicitly, so
the same seed gives the same graph on every machine.
"""
from __future__ import annotations

import dataclasses
import numpy as np

GRAPH500_ABCD = (0.57, 0.19, 0.19, 0.05)


@dataclasses.dataclass
class Graph:
    """Undirected simple graph in CSR form (each undirected edge stored twice)."""
    n: int
    row_ptr: np.ndarray   # int64 [n+1]
    col: np.ndarray       # int32 [m_dir], rows sorted ascending, no self loops
    labels: np.ndarray    # uint8 [n]
    name: str = ""

    @property
    def m_dir(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


@dataclasses.dataclass
class Template:
    """Small connected template G0: n0 vertices, labels, undirected edge list."""
    labels: list
    edges: list           # list of (a, b) with a != b, each undirected edge once
    name: str = ""

    @property
    def n0(self) -> int:
        return len(self.labels)

    @property
    def m0(self) -> int:
        return len(self.edges)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def rmat_edges(scale: int, edge_factor: int = 16, abcd=GRAPH500_ABCD,
               seed: int = 1, chunk: int = 1 << 24):
    """Draw edge_factor * 2^scale directed R-MAT edges (src, dst) as uint32.

    At every one of the `scale` levels an edge picks one quadrant with
    probabilities (A, B, C, D), D = 1 - A - B - C, with no noise.  The vertex ids
    are then relabelled by a seeded random permutation (Graph 500 style) so
    that vertex id carries no degree information.
    """
    a, b, c = abcd[0], abcd[1], abcd[2]
    n = 1 << scale
    m = edge_factor * n
    t_a = np.uint32(min(int(a * 2**32), 2**32 - 1))
    t_ab = np.uint32(min(int((a + b) * 2**32), 2**32 - 1))
    t_abc = np.uint32(min(int((a + b + c) * 2**32), 2**32 - 1))
    rng = _rng(seed)
    src = np.zeros(m, dtype=np.uint32)
    dst = np.zeros(m, dtype=np.uint32)
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        s = np.zeros(hi - lo, dtype=np.uint32)
        d = np.zeros(hi - lo, dtype=np.uint32)
        raw = None
        for level in range(scale):
            # two 32-bit draws per 64-bit Philox output
            if level % 2 == 0:
                raw = rng.bit_generator.random_raw(hi - lo)
                r = (raw & np.uint64(0xFFFFFFFF)).astype(np.uint32)
            else:
                r = (raw >> np.uint64(32)).astype(np.uint32)
            sbit = (r >= t_ab)
            dbit = ((r >= t_a) & (r < t_ab)) | (r >= t_abc)
            s |= sbit.astype(np.uint32) << np.uint32(level)
            d |= dbit.astype(np.uint32) << np.uint32(level)
        src[lo:hi] = s
        dst[lo:hi] = d
    perm = _rng(seed ^ 0x5EED).permutation(n).astype(np.uint32)
    return perm[src], perm[dst]


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, device=None):
    """Symmetrise, drop self loops, deduplicate and sort into CSR.

    `device` optionally names a torch CUDA device used only to sort the keys
    faster; the result is identical either way (a sort is exact).
    """
    keep = src != dst
    s = src[keep].astype(np.int64)
    d = dst[keep].astype(np.int64)
    keys = np.concatenate([s * n + d, d * n + s])
    del s, d
    if device is not None:
        import torch
        t = torch.from_numpy(keys).to(device)
        t = torch.unique(t, sorted=True)
        keys = t.cpu().numpy()
        del t
    else:
        keys.sort()
        if keys.shape[0]:
            keep = np.empty(keys.shape[0], dtype=bool)
            keep[0] = True
            np.not_equal(keys[1:], keys[:-1], out=keep[1:])
            keys = keys[keep]
    rows = keys // n
    col = (keys - rows * n).astype(np.int32)
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, col


def degree_labels(row_ptr: np.ndarray) -> np.ndarray:
    """l(v) = ceil(log2(d+1)) = bit length of d (0 for an isolated vertex)."""
    d = np.diff(row_ptr).astype(np.int64)
    lab = np.zeros(d.shape[0], dtype=np.uint8)
    x = d.copy()
    while np.any(x > 0):
        nz = x > 0
        lab[nz] += 1
        x >>= 1
    return lab


def zipf_labels(n: int, n_labels: int = 64, s: float = 1.2, seed: int = 7) -> np.ndarray:
    """iid labels with P(k) proportional to (k+1)^-s, k = 0..n_labels-1."""
    w = (np.arange(n_labels, dtype=np.float64) + 1.0) ** (-s)
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    u = _rng(seed).random(n)
    return np.searchsorted(cdf, u, side="right").astype(np.uint8)


def rmat_graph(scale: int, edge_factor: int = 16, abcd=GRAPH500_ABCD, seed: int = 1,
               labels: str = "degree", n_labels: int = 64, zipf_s: float = 1.2,
               label_seed: int = 7, device=None) -> Graph:
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor, abcd, seed)
    row_ptr, col = csr_from_edges(n, src, dst, device=device)
    del src, dst
    if labels == "degree":
        lab = degree_labels(row_ptr)
    elif labels == "zipf":
        lab = zipf_labels(n, n_labels, zipf_s, label_seed)
    else:
        raise ValueError(labels)
    return Graph(n, row_ptr, col, lab, name=f"rmat{scale}-{labels}")


def graph_from_edge_list(n: int, edges, labels) -> Graph:
    """Small hand-built graphs (tests): undirected edge list -> CSR."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    src = e[:, 0].astype(np.uint32)
    dst = e[:, 1].astype(np.uint32)
    row_ptr, col = csr_from_edges(n, src, dst)
    return Graph(n, row_ptr, col, np.asarray(labels, dtype=np.uint8))


def edge_labels(row_ptr, col, n_labels: int, seed: int = 3, weights=None):
    """One label per undirected edge, the same on both of its CSR entries:
    edge {x, y} (x < y) draws Philox4x32-10 with counter (y, x, 0, 0), so the
    two directions agree without a lookup.  `weights` (optional) skews the
    distribution over 0..n_labels-1.  Numpy arrays in, a uint8 numpy array
    out; torch tensors in, a uint8 tensor out on their device (same values)."""
    import torch
    on_torch = isinstance(col, torch.Tensor)
    rp = row_ptr if on_torch else torch.from_numpy(np.ascontiguousarray(row_ptr, dtype=np.int64))
    c = (col if on_torch else torch.from_numpy(np.ascontiguousarray(col))).to(torch.int64)
    rp = rp.to(torch.int64)
    n = rp.shape[0] - 1
    src = torch.repeat_interleave(torch.arange(n, device=rp.device, dtype=torch.int64), rp[1:] - rp[:-1])
    lo, hi = torch.minimum(src, c), torch.maximum(src, c)
    del src, c
    z = torch.zeros_like(lo)
    r0, _, _, _ = philox4x32(hi, lo, z, z, seed & _U32, 0x2545F491)
    del lo, hi, z
    u = r0.to(torch.float64) / 4294967296.0
    if weights is None:
        lab = torch.clamp(torch.floor(u * n_labels).to(torch.int64), max=n_labels - 1)
    else:
        w = torch.as_tensor(np.asarray(weights, dtype=np.float64), device=u.device)
        cdf = torch.cumsum(w / w.sum(), 0)
        lab = torch.clamp(torch.searchsorted(cdf, u, right=True), max=n_labels - 1)
    lab = lab.to(torch.uint8)
    return lab if on_torch else lab.numpy()


def sampled_template(g, el, n0, extra, seed):
    """A template that matches at least once: n0 vertices reached by a
    breadth-first walk from a random vertex of degree >= 2, the walk's tree
    edges plus up to `extra` more edges among them, with the graph's vertex
    and edge labels."""
    rng = np.random.default_rng(seed)
    deg = np.diff(g.row_ptr)
    starts = np.nonzero(deg >= 2)[0]
    for _ in range(100):
        root = int(rng.choice(starts))
        order, parent, seen = [root], {root: -1}, {root}
        for v in order:
            for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
                u = int(g.col[e])
                if u not in seen and len(order) < n0:
                    seen.add(u)
                    parent[u] = v
                    order.append(u)
        if len(order) == n0:
            break
    idx = {v: i for i, v in enumerate(order)}
    label_of = {}
    for v in order:
        for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
            u = int(g.col[e])
            if u in idx:
                label_of[(idx[v], idx[u])] = int(el[e]) if el is not None else 0
    edges = [(idx[parent[v]], idx[v]) for v in order[1:]]
    chords = [(a, b) for (a, b) in label_of if a < b and (a, b) not in edges and (b, a) not in edges]
    rng.shuffle(chords)
    edges += [tuple(c) for c in chords[:extra]]
    edges = [(min(a, b), max(a, b)) for a, b in edges]
    tel = [label_of[e] for e in edges]
    tl = [int(g.labels[v]) for v in order]
    return tl, edges, tel


def label_frequencies(g: Graph, n_labels: int = 256) -> np.ndarray:
    return np.bincount(g.labels, minlength=n_labels)[:n_labels].astype(np.int64)


# ---------------------------------------------------------------------------
# Templates
# ---------------------------------------------------------------------------

def is_connected(n0: int, edges) -> bool:
    adj = [set() for _ in range(n0)]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    seen = {0}
    stack = [0]
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return len(seen) == n0


def random_template(seed: int, n0: int, extra_edges: int, label_pool,
                    label_weights=None) -> Template:
    """Random connected template: a random spanning tree plus `extra_edges`
    chords, labels drawn from `label_pool` (optionally weighted)."""
    rng = _rng(seed)
    edges = set()
    for v in range(1, n0):
        u = int(rng.integers(0, v))
        edges.add((u, v))
    possible = [(a, b) for a in range(n0) for b in range(a + 1, n0) if (a, b) not in edges]
    rng.shuffle(possible)
    for e in possible[:extra_edges]:
        edges.add(tuple(e))
    pool = np.asarray(label_pool)
    p = None
    if label_weights is not None:
        p = np.asarray(label_weights, dtype=np.float64)
        p = p / p.sum()
    labs = [int(x) for x in rng.choice(pool, size=n0, p=p)]
    return Template(labs, sorted(edges), name=f"rand{seed}")


def edit_variants(base: Template, count: int, seed: int, label_pool,
                  max_k: int = 2, n_min: int = 5, n_max: int = 9):
    """Edit-distance variants of `base` for the exploratory-search workload
    (Section 6.7): each variant applies k in {1, 2} random edits drawn from
    {delete an edge keeping the template connected, add an edge, delete a
    leaf, add a leaf}.  Variants keep 5..9 vertices; duplicates are allowed."""
    rng = _rng(seed)
    out = []
    tries = 0
    while len(out) < count and tries < count * 200:
        tries += 1
        labels = list(base.labels)
        edges = set(tuple(sorted(e)) for e in base.edges)
        k = int(rng.integers(1, max_k + 1))
        ok = True
        for _ in range(k):
            op = int(rng.integers(0, 4))
            n0 = len(labels)
            if op == 0:     # delete an edge, keep connected
                cand = sorted(edges)
                rng.shuffle(cand)
                done = False
                for e in cand:
                    trial = edges - {e}
                    if is_connected(n0, trial):
                        edges = trial
                        done = True
                        break
                ok &= done
            elif op == 1:   # add an edge
                cand = [(a, b) for a in range(n0) for b in range(a + 1, n0) if (a, b) not in edges]
                if not cand:
                    ok = False
                    break
                edges.add(cand[int(rng.integers(0, len(cand)))])
            elif op == 2:   # delete a leaf
                deg = [0] * n0
                for a, b in edges:
                    deg[a] += 1
                    deg[b] += 1
                leaves = [v for v in range(n0) if deg[v] == 1]
                if not leaves or n0 <= n_min:
                    ok = False
                    break
                x = leaves[int(rng.integers(0, len(leaves)))]
                edges = set((a - (a > x), b - (b > x)) for a, b in edges if x not in (a, b))
                labels = labels[:x] + labels[x + 1:]
            else:           # add a leaf
                if n0 >= n_max:
                    ok = False
                    break
                u = int(rng.integers(0, n0))
                labels.append(int(label_pool[int(rng.integers(0, len(label_pool)))]))
                edges.add((u, n0))
        if not ok:
            continue
        n0 = len(labels)
        if not (n_min <= n0 <= n_max) or not is_connected(n0, edges):
            continue
        out.append(Template(labels, sorted(edges), name=f"{base.name}-ed{len(out)}"))
    return out


def labels_by_frequency(g: Graph):
    """Labels sorted from most to least frequent (ties: smaller label first)."""
    f = label_frequencies(g)
    order = sorted(range(len(f)), key=lambda L: (-f[L], L))
    return [L for L in order if f[L] > 0]


# ---------------------------------------------------------------------------
# Large graphs generated where they are used (scale 20-25)
#
# The numpy recipe above draws on one host core; at scales 24-25 (2.7-5.4e8
# draws of `scale` quadrant choices each) that takes minutes.  The recipe below
# is the same R-MAT process written as integer torch operations, so it runs on
# a CUDA device in seconds and gives bit-identical arrays on the CPU (tests
# check this at small scales).  Its random numbers come from Philox4x32-10
# (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2,
# 3", SC 2011), a counter-based generator: word j of draw block b of item i is
# a pure function of (i, stream, b, seed), so chunks can be generated in any
# order.  Each R-MAT level uses a 16-bit draw (two levels per 32-bit word);
# the quadrant thresholds are the (A, B, C) cumulative probabilities rounded to
# multiples of 2^-16.
# ---------------------------------------------------------------------------

_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57      # round multipliers
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85      # Weyl key increments
_U32 = 0xFFFFFFFF

# Philox streams (third counter word) of the different draws
_S_EDGE, _S_PERM, _S_LABEL = 1, 2, 3


def _mulhilo32(m: int, x):
    """(hi, lo) 32-bit halves of the 64-bit product m * x, for a constant
    m < 2^32 and an int64 tensor x of values in [0, 2^32).  The constant is
    split into 16-bit halves so that no intermediate leaves int64."""
    mh, ml = m >> 16, m & 0xFFFF
    a = x * mh                                   # < 2^48
    b = ((a & 0xFFFF) << 16) + x * ml            # < 2^49
    return (a >> 16) + (b >> 32), b & _U32


def philox4x32(c0, c1, c2, c3, k0: int, k1: int, rounds: int = 10):
    """Philox4x32-R on int64 tensors holding 32-bit counter words (any shape,
    broadcast together); key (k0, k1).  Returns the four 32-bit output words
    as int64 tensors."""
    import torch
    x0, x1, x2, x3 = torch.broadcast_tensors(c0, c1, c2, c3)
    x0, x1, x2, x3 = x0.clone(), x1.clone(), x2.clone(), x3.clone()
    for r in range(rounds):
        if r:
            k0 = (k0 + _PHILOX_W0) & _U32
            k1 = (k1 + _PHILOX_W1) & _U32
        hi0, lo0 = _mulhilo32(_PHILOX_M0, x0)
        hi1, lo1 = _mulhilo32(_PHILOX_M1, x2)
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return x0, x1, x2, x3


def _draw_words(idx, stream: int, block: int, seed: int):
    """Four 32-bit Philox words for every item index in `idx` (int64 tensor)."""
    import torch
    lo = idx & _U32
    hi = idx >> 32
    c2 = torch.full_like(idx, stream)
    c3 = torch.full_like(idx, block)
    return philox4x32(lo, hi, c2, c3, seed & _U32, (seed >> 32) & _U32)


@dataclasses.dataclass
class DeviceGraph:
    """CSR graph held as torch tensors (on any device): row_ptr int64 [n+1],
    col int32 [m_dir], labels uint8 [n]."""
    n: int
    row_ptr: object
    col: object
    labels: object
    name: str = ""

    @property
    def m_dir(self) -> int:
        return int(self.col.shape[0])

    def to_host(self) -> Graph:
        return Graph(self.n, self.row_ptr.cpu().numpy(), self.col.cpu().numpy(),
                     self.labels.cpu().numpy(), name=self.name)


def rmat_edges_philox(scale: int, edge_factor: int = 16, abcd=GRAPH500_ABCD, seed: int = 1,
                      device="cpu", chunk: int = 1 << 24):
    """edge_factor * 2^scale directed R-MAT draws (src, dst), int64 tensors on
    `device`, vertex ids relabelled by a seeded random permutation."""
    import torch
    n = 1 << scale
    m = edge_factor * n
    t_a = int(round(abcd[0] * 65536))
    t_ab = int(round((abcd[0] + abcd[1]) * 65536))
    t_abc = int(round((abcd[0] + abcd[1] + abcd[2]) * 65536))
    # permutation: stable sort of 64-bit random keys (ties impossible to
    # matter: a stable sort of equal keys keeps index order)
    vid = torch.arange(n, dtype=torch.int64, device=device)
    w = _draw_words(vid, _S_PERM, 0, seed)
    pkey = (w[0] << 31) | (w[1] >> 1)
    perm = torch.argsort(pkey, stable=True)
    del vid, w, pkey
    srcs, dsts = [], []
    for lo in range(0, m, chunk):
        hi = min(m, lo + chunk)
        idx = torch.arange(lo, hi, dtype=torch.int64, device=device)
        s = torch.zeros_like(idx)
        d = torch.zeros_like(idx)
        words = None
        for level in range(scale):
            if level % 8 == 0:
                words = _draw_words(idx, _S_EDGE, level // 8, seed)
            wd = words[(level % 8) // 2]
            r = (wd >> 16) if (level & 1) else (wd & 0xFFFF)
            sbit = r >= t_ab
            dbit = ((r >= t_a) & (r < t_ab)) | (r >= t_abc)
            s |= sbit.to(torch.int64) << level
            d |= dbit.to(torch.int64) << level
        srcs.append(perm[s])
        dsts.append(perm[d])
        del idx, s, d, words
    return torch.cat(srcs), torch.cat(dsts)


def csr_from_edges_torch(n: int, src, dst):
    """Symmetrise, drop self loops, deduplicate and sort into CSR (torch, any
    device); returns (row_ptr int64 [n+1], col int32 [m_dir])."""
    import torch
    keep = src != dst
    s, d = src[keep], dst[keep]
    del keep
    keys = torch.cat([s * n + d, d * n + s])
    del s, d
    keys = torch.unique(keys, sorted=True)
    rows = torch.div(keys, n, rounding_mode="floor")
    col = (keys - rows * n).to(torch.int32)
    del keys
    counts = torch.bincount(rows, minlength=n)
    del rows
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=col.device)
    torch.cumsum(counts, 0, out=row_ptr[1:])
    return row_ptr, col


def zipf_labels_philox(n: int, n_labels: int = 64, s: float = 1.2, seed: int = 7, device="cpu"):
    """iid labels with P(k) proportional to (k+1)^-s: a uniform 32-bit Philox
    word per vertex, looked up in the float64 cumulative distribution."""
    import torch
    w = (np.arange(n_labels, dtype=np.float64) + 1.0) ** (-s)
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    cdf_t = torch.from_numpy(cdf).to(device)
    vid = torch.arange(n, dtype=torch.int64, device=device)
    u = _draw_words(vid, _S_LABEL, 0, seed)[0].to(torch.float64) * (1.0 / 4294967296.0)
    return torch.searchsorted(cdf_t, u, right=True).to(torch.uint8)


def degree_labels_torch(row_ptr):
    """Bit length of every degree (0 for an isolated vertex), uint8."""
    import torch
    x = row_ptr[1:] - row_ptr[:-1]
    lab = torch.zeros(x.shape[0], dtype=torch.uint8, device=x.device)
    while bool((x > 0).any()):
        lab += (x > 0).to(torch.uint8)
        x = x >> 1
    return lab


def rmat_graph_philox(scale: int, edge_factor: int = 16, abcd=GRAPH500_ABCD, seed: int = 1,
                      labels: str = "zipf", n_labels: int = 64, zipf_s: float = 1.2,
                      label_seed: int = 7, device="cpu") -> DeviceGraph:
    """R-MAT graph with the Philox recipe, built on `device` (a CUDA device at
    scales 20-25; the CPU gives the same arrays, slowly)."""
    import torch
    n = 1 << scale
    with torch.no_grad():
        src, dst = rmat_edges_philox(scale, edge_factor, abcd, seed, device=device)
        row_ptr, col = csr_from_edges_torch(n, src, dst)
        del src, dst
        if labels == "degree":
            lab = degree_labels_torch(row_ptr)
        elif labels == "zipf":
            lab = zipf_labels_philox(n, n_labels, zipf_s, label_seed, device=device)
        else:
            raise ValueError(labels)
    return DeviceGraph(n, row_ptr, col, lab, name=f"rmat{scale}-{labels}-philox")
