"""CPU oracle for the constraint-checking pipeline -- TEST INFRASTRUCTURE.

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline /
reference leg may import this package.  The product (the CUDA library and its
binding) never does, and it shares no code with it.

* `ccpm_oracle.c`  -- plain single-threaded C: init (Alg. 3), one LCC round and
  the LCC fixpoint (Alg. 4/5), one NLCC constraint (Alg. 6/7, as an injective
  rooted-embedding search), final template-driven search with match counting
  (Remark 1, Section 4.7), and the listing of every match with per-vertex and
  per-entry participation counts (the analyses of the Introduction).
* `constraints.py` -- non-local constraint generation (Table 3, Alg. 2).
* `pipeline.py`    -- the main loop (Alg. 1) over the pieces above.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccpm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_libs = {}


def build(force: bool = False) -> str:
    """Compile the C oracle in place with gcc -O2: liboracle.so runs on one
    thread (the pragmas are ignored), liboracle_omp.so with OpenMP runs the
    loops the source marks as independent on every host core."""
    for path, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
            tmp = path + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wno-unknown-pragmas"] + extra +
                                  ["-o", tmp, _SRC])
            os.replace(tmp, path)
    return _LIB


def threads() -> int:
    """Threads the OpenMP build uses (OMP_NUM_THREADS, else every core)."""
    env = os.environ.get("OMP_NUM_THREADS")
    return int(env) if env else (os.cpu_count() or 1)


_parallel = False


def set_parallel(on: bool) -> None:
    """Route every oracle call through the OpenMP build (True) or the
    single-threaded one (False, the default).  Results are identical."""
    global _parallel
    _parallel = bool(on)


def lib():
    key = "omp" if _parallel else "serial"
    if key not in _libs:
        build()
        L = ctypes.CDLL(_LIB_OMP if _parallel else _LIB)
        i64, i32, u32p = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        vp = ctypes.c_void_p
        L.oracle_init.argtypes = [i64, vp, vp, vp, i32, vp, vp, vp]
        L.oracle_init.restype = None
        L.oracle_lcc_round.argtypes = [i64, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_lcc_round.restype = ctypes.c_int
        L.oracle_lcc.argtypes = [i64, vp, vp, i32, vp, vp, vp, vp, vp]
        L.oracle_lcc.restype = ctypes.c_int64
        L.oracle_nlcc.argtypes = [i64, vp, vp, ctypes.c_uint32, vp, ctypes.c_uint32, vp, vp, vp, vp]
        L.oracle_nlcc.restype = ctypes.c_int
        L.oracle_final.argtypes = [i64, vp, vp, i32, vp, i32, vp, vp, vp, vp, vp, vp, ctypes.c_uint64, vp]
        L.oracle_final.restype = ctypes.c_int
        L.oracle_matches.argtypes = [i64, vp, vp, i32, vp, i32, vp, vp, vp, vp, ctypes.c_uint64, vp, vp]
        L.oracle_matches.restype = ctypes.c_uint64
        L.oracle_wide_init.argtypes = [i64, vp, vp, vp, i32, vp, vp, vp]
        L.oracle_wide_init.restype = None
        L.oracle_wide_lcc_round.argtypes = [i64, vp, vp, vp, i32, vp, i32, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_wide_lcc_round.restype = ctypes.c_int
        L.oracle_wide_lcc.argtypes = [i64, vp, vp, vp, vp, i32, vp, i32, vp, vp, vp, vp, vp]
        L.oracle_wide_lcc.restype = ctypes.c_int64
        _libs[key] = L
    return _libs[key]


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def template_tables(labels, edges):
    n0 = len(labels)
    tlab = np.zeros(32, dtype=np.uint8)
    tlab[:n0] = labels
    tadj = np.zeros(32, dtype=np.uint32)
    for a, b in edges:
        tadj[a] |= np.uint32(1 << b)
        tadj[b] |= np.uint32(1 << a)
    return tlab, tadj


class Graph:
    """Contiguous views of a CSR graph as the C oracle wants them."""

    def __init__(self, row_ptr, col, labels):
        self.rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.lab = np.ascontiguousarray(labels, dtype=np.uint8)
        self.n = int(self.rp.shape[0] - 1)
        self.m = int(self.rp[-1])


def init(g: Graph, labels, edges):
    tlab, _ = template_tables(labels, edges)
    omega = np.zeros(max(g.n, 1), dtype=np.uint32)[: g.n]
    A = np.zeros(max(g.m, 1), dtype=np.uint8)[: g.m]
    omega = np.ascontiguousarray(omega)
    A = np.ascontiguousarray(A)
    lib().oracle_init(g.n, _p(g.rp), _p(g.col), _p(g.lab), len(labels), _p(tlab), _p(omega), _p(A))
    return omega, A


def lcc_round(g: Graph, labels, edges, omega, A):
    """One Jacobi LCC round.  Returns (changed, omega', A', scanned)."""
    tlab, tadj = template_tables(labels, edges)
    om2 = np.zeros_like(omega)
    A2 = np.zeros_like(A)
    sc = np.zeros(1, dtype=np.int64)
    ch = lib().oracle_lcc_round(g.n, _p(g.rp), _p(g.col), len(labels), _p(tlab), _p(tadj),
                                _p(omega), _p(A), _p(om2), _p(A2), _p(sc))
    return bool(ch), om2, A2, int(sc[0])


def lcc(g: Graph, labels, edges, omega, A):
    """LCC to fixpoint in place.  Returns (rounds, scanned)."""
    tlab, tadj = template_tables(labels, edges)
    sc = np.zeros(1, dtype=np.int64)
    r = lib().oracle_lcc(g.n, _p(g.rp), _p(g.col), len(labels), _p(tlab), _p(tadj),
                         _p(omega), _p(A), _p(sc))
    if r < 0:
        raise MemoryError("oracle_lcc")
    return int(r), int(sc[0])


def nlcc(g: Graph, svert_mask: int, sadj, heads_mask: int, omega, A, with_scanned=False):
    """One non-local constraint in place.  Returns (changed, tokens issued[,
    CSR entries examined])."""
    sadj = np.ascontiguousarray(np.asarray(list(sadj) + [0] * (32 - len(sadj)), dtype=np.uint32))
    nt = np.zeros(1, dtype=np.int64)
    ns = np.zeros(1, dtype=np.int64)
    ch = lib().oracle_nlcc(g.n, _p(g.rp), _p(g.col), svert_mask, _p(sadj), heads_mask,
                           _p(omega), _p(A), _p(nt), _p(ns))
    if ch < 0:
        raise MemoryError("oracle_nlcc")
    if with_scanned:
        return bool(ch), int(nt[0]), int(ns[0])
    return bool(ch), int(nt[0])


def final(g: Graph, labels, edges, omega, A, cap: int, with_scanned=False):
    """Full template-driven search.  Returns (status, omega*, A*, count[,
    CSR entries examined])."""
    _, tadj = template_tables(labels, edges)
    te = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    om2 = np.zeros_like(omega)
    A2 = np.zeros_like(A)
    cnt = np.zeros(1, dtype=np.uint64)
    ns = np.zeros(1, dtype=np.int64)
    st = lib().oracle_final(g.n, _p(g.rp), _p(g.col), len(labels), _p(tadj), len(edges), _p(te),
                            _p(omega), _p(A), _p(om2), _p(A2), _p(cnt), int(cap), _p(ns))
    if with_scanned:
        return int(st), om2, A2, int(cnt[0]), int(ns[0])
    return int(st), om2, A2, int(cnt[0])


def matches(g: Graph, labels, edges, omega, A, list_cap: int = 0):
    """Every match inside (omega, A): (count, list [min(count, list_cap), n0]
    int32, per-vertex counts uint64 [n], per-entry counts uint64 [m])."""
    _, tadj = template_tables(labels, edges)
    n0 = len(labels)
    te = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    lst = np.zeros((max(list_cap, 1), n0), dtype=np.int32)
    vc = np.zeros(max(g.n, 1), dtype=np.uint64)
    ec = np.zeros(max(g.m, 1), dtype=np.uint64)
    cnt = lib().oracle_matches(g.n, _p(g.rp), _p(g.col), n0, _p(tadj), len(edges), _p(te),
                               _p(omega), _p(A), _p(lst), int(list_cap), _p(vc), _p(ec))
    return int(cnt), lst[: min(int(cnt), list_cap)], vc[: g.n], ec[: g.m]


def pack_bits(A: np.ndarray) -> np.ndarray:
    """Byte-per-entry edge flags -> uint32 words, bit e&31 of word e>>5."""
    m = A.shape[0]
    words = (m + 31) // 32
    b = np.packbits(A.astype(np.uint8), bitorder="little")
    out = np.zeros(words * 4, dtype=np.uint8)
    out[: b.shape[0]] = b
    return out.view("<u4").astype(np.uint32)


# --------------------------------------------------------------------------
# Wider templates (n0 <= 64, 64-bit omega) and edge labels: the LCC phase.


def _wide_template(labels, edges, edge_labels):
    n0 = len(labels)
    assert 2 <= n0 <= 64
    tlab = np.zeros(64, dtype=np.uint8)
    tlab[:n0] = labels
    te = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    if te.size == 0:
        te = np.zeros(2, dtype=np.int32)
    tel = None
    if edge_labels is not None:
        tel = np.ascontiguousarray(np.asarray(edge_labels, dtype=np.uint8))
        assert tel.shape[0] == len(edges)
    return n0, tlab, te, tel


def _opt(a):
    return None if a is None else _p(a)


def wide_init(g: Graph, labels):
    n0 = len(labels)
    tlab = np.zeros(64, dtype=np.uint8)
    tlab[:n0] = labels
    omega = np.ascontiguousarray(np.zeros(max(g.n, 1), dtype=np.uint64)[: g.n])
    A = np.ascontiguousarray(np.zeros(max(g.m, 1), dtype=np.uint8)[: g.m])
    lib().oracle_wide_init(g.n, _p(g.rp), _p(g.col), _p(g.lab), n0, _p(tlab), _p(omega), _p(A))
    return omega, A


def wide_lcc_round(g: Graph, labels, edges, omega, A, edge_labels=None, graph_edge_labels=None):
    """One snapshot round with 64-bit omega and edge labels.
    Returns (changed, omega', A', scanned)."""
    n0, tlab, te, tel = _wide_template(labels, edges, edge_labels)
    el = None if graph_edge_labels is None else np.ascontiguousarray(graph_edge_labels, dtype=np.uint8)
    om2 = np.zeros_like(omega)
    A2 = np.zeros_like(A)
    sc = np.zeros(1, dtype=np.int64)
    ch = lib().oracle_wide_lcc_round(g.n, _p(g.rp), _p(g.col), _opt(el), n0, _p(tlab), len(edges), _p(te),
                                     _opt(tel), _p(omega), _p(A), _p(om2), _p(A2), _p(sc))
    if ch < 0:
        raise MemoryError("oracle_wide_lcc_round")
    return bool(ch), om2, A2, int(sc[0])


def wide_lcc(g: Graph, labels, edges, edge_labels=None, graph_edge_labels=None):
    """Init and LCC to its fixpoint with 64-bit omega and edge labels.
    Returns (omega uint64[n], A uint8[m], rounds, scanned)."""
    n0, tlab, te, tel = _wide_template(labels, edges, edge_labels)
    el = None if graph_edge_labels is None else np.ascontiguousarray(graph_edge_labels, dtype=np.uint8)
    omega = np.ascontiguousarray(np.zeros(max(g.n, 1), dtype=np.uint64)[: g.n])
    A = np.ascontiguousarray(np.zeros(max(g.m, 1), dtype=np.uint8)[: g.m])
    sc = np.zeros(1, dtype=np.int64)
    r = lib().oracle_wide_lcc(g.n, _p(g.rp), _p(g.col), _p(g.lab), _opt(el), n0, _p(tlab), len(edges), _p(te),
                              _opt(tel), _p(omega), _p(A), _p(sc))
    if r < 0:
        raise MemoryError("oracle_wide_lcc")
    return omega, A, int(r), int(sc[0])
