"""Main constraint-checking loop of the oracle (Alg. 1) -- TEST INFRASTRUCTURE.

init (Alg. 3) -> LCC to fixpoint (Alg. 4) -> for each non-local constraint in
order: NLCC (Alg. 6/7), and LCC again if any omega changed (Alg. 1) -> final
template-driven search over the full template, which also counts matches
(Remark 1; Section 4.7).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import Graph, init, lcc, nlcc, final, pack_bits
from . import constraints as cgen

DEFAULT_MAX_EMBEDDINGS = 1 << 32


@dataclasses.dataclass
class OracleResult:
    omega: np.ndarray            # uint32 [n]
    A: np.ndarray                # uint8 [m_dir] (byte per CSR entry)
    ebits: np.ndarray            # uint32 words, bit e&31 of word e>>5
    phase_rounds: list           # LCC rounds per phase: [initial, after C1, after C2, ...]
    nlcc_changed: list           # per constraint: did it change omega
    match_embeddings: int
    count_valid: bool
    automorphisms: int
    active_v: int
    active_e_dir: int
    lcc_scanned: int             # sum over rounds of active entries at round start
    tokens: int
    search_scanned: int = 0      # CSR entries examined by the searches (metric only)
    seconds: float = 0.0
    omega_pre_final: np.ndarray = None
    A_pre_final: np.ndarray = None

    @property
    def lcc_rounds_total(self) -> int:
        return int(sum(self.phase_rounds))

    @property
    def match_subgraphs(self) -> int:
        return self.match_embeddings // self.automorphisms if self.automorphisms else 0


def automorphisms(labels, edges) -> int:
    """Label-preserving automorphisms of the template, by plain backtracking."""
    n0 = len(labels)
    adj = [[False] * n0 for _ in range(n0)]
    for a, b in edges:
        adj[a][b] = adj[b][a] = True
    img = [-1] * n0
    used = [False] * n0

    def rec(i):
        if i == n0:
            return 1
        total = 0
        for x in range(n0):
            if used[x] or labels[x] != labels[i]:
                continue
            if any(adj[i][j] != adj[x][img[j]] for j in range(i)):
                continue
            img[i] = x
            used[x] = True
            total += rec(i + 1)
            used[x] = False
        img[i] = -1
        return total

    return rec(0)


def run(row_ptr, col, labels, tlabels, tedges, constraints=None,
        max_embeddings: int = DEFAULT_MAX_EMBEDDINGS) -> OracleResult:
    """Whole pipeline.  `constraints` is an ordered list of oracle Constraint
    objects (default: the oracle's own Table 3 generation)."""
    t0 = time.perf_counter()
    g = Graph(row_ptr, col, labels)
    tlabels = [int(x) for x in tlabels]
    tedges = [(int(a), int(b)) for a, b in tedges]
    if constraints is None:
        constraints = cgen.generate(tlabels, tedges)
    omega, A = init(g, tlabels, tedges)
    r, scanned = lcc(g, tlabels, tedges, omega, A)
    phase = [r]
    changed_list = []
    tokens = 0
    search_scanned = 0
    for c in constraints:
        ch, nt, ns = nlcc(g, c.vmask(), c.sadj(len(tlabels)), c.hmask(), omega, A, with_scanned=True)
        tokens += nt
        search_scanned += ns
        changed_list.append(ch)
        if ch:
            r, sc = lcc(g, tlabels, tedges, omega, A)
            scanned += sc
        else:
            r = 0
        phase.append(r)
    om_pre, A_pre = omega.copy(), A.copy()
    st, om_f, A_f, count, ns = final(g, tlabels, tedges, omega, A, max_embeddings, with_scanned=True)
    search_scanned += ns
    valid = st == 0
    omega, A = om_f, A_f          # exact even when the count ran past its cap
    res = OracleResult(
        omega=omega, A=A, ebits=pack_bits(A), phase_rounds=phase,
        nlcc_changed=changed_list, match_embeddings=count if valid else 0,
        count_valid=valid, automorphisms=automorphisms(tlabels, tedges),
        active_v=int(np.count_nonzero(omega)), active_e_dir=int(np.count_nonzero(A)),
        lcc_scanned=scanned, tokens=tokens, search_scanned=search_scanned, omega_pre_final=om_pre, A_pre_final=A_pre)
    res.seconds = time.perf_counter() - t0
    return res
