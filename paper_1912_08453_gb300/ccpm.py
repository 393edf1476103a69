"""Thin ctypes binding of the C ABI in include/ccpm.h.

Argument marshalling only: every step of the pruning pipeline runs in the CUDA
library `libccpm.so`.  There is no CPU fallback; if the library is missing the
import of this module fails with a RuntimeError.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); CUDA tensors are passed as borrowed device pointers.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libccpm.so")

CCPM_OK, CCPM_EINVAL, CCPM_ENOMEM, CCPM_ECUDA = 0, 1, 2, 3
CCPM_ETIMEOUT, CCPM_EOVERFLOW, CCPM_EBUDGET, CCPM_ESTATE = 4, 5, 6, 7
CCPM_HOST_PTRS, CCPM_DEVICE_PTRS, CCPM_VALIDATE = 0, 1, 2
CCPM_ORDER_FIXED, CCPM_ORDER_EXPLICIT, CCPM_ORDER_LEARNED = 0, 1, 2
MLP_IN, MLP_HIDDEN = 16, 64
MLP_PARAMS = MLP_IN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN + 1
KIND_NAMES = {0: "PC", 1: "CC", 2: "TDS_CC", 3: "TDS_PC", 4: "TDS"}
MAX_TMPL_EDGES = 496


class CcpmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ccpm error {code}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("order_mode", ctypes.c_int), ("run_final", ctypes.c_int),
                ("max_embeddings", ctypes.c_uint64), ("search_budget", ctypes.c_uint64),
                ("hub_degree", ctypes.c_int), ("batch_workers", ctypes.c_int), ("resume", ctypes.c_int),
                ("compact", ctypes.c_int), ("search_split", ctypes.c_int),
                ("lcc_only", ctypes.c_int), ("short_rows", ctypes.c_int), ("no_edge_elimination", ctypes.c_int),
                ("entry_labels", ctypes.c_int), ("grid_share", ctypes.c_int),
                ("mlp", ctypes.c_void_p)]


class WideStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("edges_scanned", ctypes.c_int64),
                ("vertices_scanned", ctypes.c_int64), ("active_v", ctypes.c_int64),
                ("active_e_dir", ctypes.c_int64), ("ms", ctypes.c_double)]


class Counts(ctypes.Structure):
    _fields_ = [("active_v", ctypes.c_int64), ("active_e_dir", ctypes.c_int64),
                ("lcc_rounds_total", ctypes.c_int64), ("n_phases", ctypes.c_int32),
                ("nlcc_constraints_run", ctypes.c_int32), ("match_embeddings", ctypes.c_uint64),
                ("automorphisms", ctypes.c_uint64), ("match_subgraphs", ctypes.c_uint64),
                ("count_valid", ctypes.c_int32), ("status", ctypes.c_int32),
                ("tokens", ctypes.c_int64), ("edges_scanned_lcc", ctypes.c_int64),
                ("edges_scanned_search", ctypes.c_int64), ("ms_total", ctypes.c_double),
                ("ms_lcc", ctypes.c_double), ("ms_nlcc", ctypes.c_double), ("ms_final", ctypes.c_double),
                ("lcc_launches", ctypes.c_int64), ("ms_lcc_kernel", ctypes.c_double),
                ("lcc_alg_bytes", ctypes.c_int64), ("lcc_row_entries", ctypes.c_int64),
                ("lcc_active_vertices", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("lcc_compactions", ctypes.c_int64), ("ms_search_kernel", ctypes.c_double),
                ("search_launches", ctypes.c_int64), ("search_entries_nlcc", ctypes.c_int64),
                ("lcc_kernel_bytes", ctypes.c_int64), ("lcc_first_entries", ctypes.c_int64),
                ("ms_lcc_first", ctypes.c_double), ("ms_final_count", ctypes.c_double),
                ("ms_final_vertex", ctypes.c_double), ("ms_final_edge", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ConstraintLog(ctypes.Structure):
    _fields_ = [("constraint", ctypes.c_int32), ("position", ctypes.c_int32),
                ("features", ctypes.c_float * MLP_IN), ("bits_before", ctypes.c_int64),
                ("bits_after", ctypes.c_int64), ("lcc_rounds", ctypes.c_int32), ("tokens", ctypes.c_int32),
                ("ms_search", ctypes.c_double), ("ms_lcc", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["features"] = list(self.features)
        return d


class ExploreVariant(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("n_edges", ctypes.c_int32), ("removed", ctypes.c_uint64),
                ("active_v", ctypes.c_int64), ("active_e_dir", ctypes.c_int64),
                ("match_embeddings", ctypes.c_uint64), ("count_valid", ctypes.c_int32),
                ("status", ctypes.c_int32), ("ms_total", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ConstraintInfo(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_verts", ctypes.c_int), ("vert_mask", ctypes.c_uint32),
                ("head_mask", ctypes.c_uint32), ("n_edges", ctypes.c_int),
                ("edges", (ctypes.c_int32 * 2) * MAX_TMPL_EDGES)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_1912_08453_gb300.build.build()")
    L = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "ccpm_ctx_create": ([i32, vp, P(vp)], i32),
        "ccpm_ctx_destroy": ([vp], None),
        "ccpm_last_error": ([vp], ctypes.c_char_p),
        "ccpm_options_default": ([P(Options)], None),
        "ccpm_graph_load_csr": ([vp, i64, i64, vp, vp, vp, i32, P(vp)], i32),
        "ccpm_graph_destroy": ([vp], None),
        "ccpm_tmpl_load": ([vp, i32, vp, i32, vp, P(vp)], i32),
        "ccpm_tmpl_destroy": ([vp], None),
        "ccpm_constraints_generate": ([vp, vp, P(i32)], i32),
        "ccpm_constraints_describe": ([vp, i32, P(ConstraintInfo)], i32),
        "ccpm_tmpl_set_order": ([vp, i32, vp], i32),
        "ccpm_prune": ([vp, vp, vp, P(Options), P(vp)], i32),
        "ccpm_prune_batch": ([vp, vp, i32, P(vp), P(Options), P(vp)], i32),
        "ccpm_result_omega": ([vp, vp, i64, i32], i32),
        "ccpm_result_edge_bitmap": ([vp, vp, i64, i32], i32),
        "ccpm_result_counts": ([vp, P(Counts)], i32),
        "ccpm_result_phase_rounds": ([vp, vp, i32], i32),
        "ccpm_result_omega_device": ([vp], vp),
        "ccpm_result_edge_bitmap_device": ([vp], vp),
        "ccpm_result_destroy": ([vp], None),
        "ccpm_result_constraint_log": ([vp, i32, P(ConstraintLog)], i32),
        "ccpm_mlp_create": ([vp, ctypes.c_uint64, P(vp)], i32),
        "ccpm_mlp_destroy": ([vp], None),
        "ccpm_mlp_set_params": ([vp, vp], i32),
        "ccpm_mlp_get_params": ([vp, vp], i32),
        "ccpm_mlp_forward": ([vp, i32, vp, vp], i32),
        "ccpm_mlp_gradient": ([vp, i32, vp, vp, vp, P(ctypes.c_float)], i32),
        "ccpm_mlp_train": ([vp, i32, vp, vp, i32, i32, ctypes.c_float, ctypes.c_uint64, P(ctypes.c_float)], i32),
        "ccpm_graph_batch_workers": ([vp], i32),
        "ccpm_graph_batch_tuning": ([vp, P(i32), P(i32), P(i32), P(i32), P(i32), P(ctypes.c_double)], i32),
        "ccpm_result_matches": ([vp, vp, vp, P(Options), vp, ctypes.c_uint64, vp, vp, i32,
                                 P(ctypes.c_uint64)], i32),
        "ccpm_explore": ([vp, vp, vp, i32, P(Options), P(ExploreVariant), i32, P(i32), P(i32),
                          P(ctypes.c_double), P(vp)], i32),
        "ccpm_state_export": ([vp, vp, P(ctypes.c_size_t)], i32),
        "ccpm_state_import": ([vp, vp, vp, vp, ctypes.c_size_t, P(vp)], i32),
        "ccpm_graph_set_edge_labels": ([vp, vp, i32], i32),
        "ccpm_lcc_wide": ([vp, vp, i32, vp, i32, vp, vp, vp, vp, i32, P(WideStats)], i32),
        "ccpm_lcc_fixpoint_noalloc": ([i32, vp, i64, i64, vp, vp, vp, i32, vp, i32, vp, vp, vp,
                                       P(ctypes.c_int32), P(ctypes.c_int64), ctypes.c_char_p, ctypes.c_size_t], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()

# every function the header declares (tests check the library exports them)
EXPORTED = ["ccpm_ctx_create", "ccpm_ctx_destroy", "ccpm_last_error", "ccpm_options_default",
            "ccpm_graph_load_csr", "ccpm_graph_destroy", "ccpm_tmpl_load", "ccpm_tmpl_destroy",
            "ccpm_constraints_generate", "ccpm_constraints_describe", "ccpm_tmpl_set_order",
            "ccpm_prune", "ccpm_prune_batch", "ccpm_result_omega", "ccpm_result_edge_bitmap", "ccpm_result_counts",
            "ccpm_result_phase_rounds", "ccpm_result_omega_device",
            "ccpm_result_edge_bitmap_device", "ccpm_result_destroy", "ccpm_lcc_fixpoint_noalloc",
            "ccpm_result_constraint_log", "ccpm_mlp_create", "ccpm_mlp_destroy", "ccpm_mlp_set_params",
            "ccpm_mlp_get_params", "ccpm_mlp_forward", "ccpm_mlp_gradient", "ccpm_mlp_train",
            "ccpm_state_export", "ccpm_state_import", "ccpm_graph_batch_workers", "ccpm_result_matches", "ccpm_explore",
            "ccpm_graph_batch_tuning", "ccpm_graph_set_edge_labels", "ccpm_lcc_wide"]


def _ptr(a):
    """(pointer, on_device) for a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(a.ctypes.data), False
    import torch
    if isinstance(a, torch.Tensor):
        assert a.is_contiguous()
        return ctypes.c_void_p(a.data_ptr()), a.is_cuda
    raise TypeError(type(a))


def options(**kw) -> Options:
    o = Options()
    lib.ccpm_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Context:
    def __init__(self, device: int = 0, stream=None):
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(int(stream)) if stream is not None else None
        rc = lib.ccpm_ctx_create(device, s, ctypes.byref(h))
        if rc:
            raise CcpmError(rc, f"ccpm_ctx_create(device={device}) failed")
        self.h = h
        self.device = device

    def check(self, rc, what=""):
        if rc:
            raise CcpmError(rc, f"{what}: {lib.ccpm_last_error(self.h).decode()}")

    def close(self):
        if self.h:
            lib.ccpm_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A resident background graph (CSR + labels) on the context's device."""

    def __init__(self, ctx: Context, row_ptr, col, labels, validate: bool = False):
        p_rp, d0 = _ptr(row_ptr)
        p_col, d1 = _ptr(col)
        p_lab, d2 = _ptr(labels)
        if not (d0 == d1 == d2):
            raise ValueError("row_ptr, col and labels must all be host or all device arrays")
        flags = CCPM_DEVICE_PTRS if d0 else CCPM_HOST_PTRS
        if validate:
            flags |= CCPM_VALIDATE
        n = int(row_ptr.shape[0]) - 1
        m = int(col.shape[0])
        h = ctypes.c_void_p()
        ctx.check(lib.ccpm_graph_load_csr(ctx.h, n, m, p_rp, p_col, p_lab, flags, ctypes.byref(h)),
                  "ccpm_graph_load_csr")
        self.h, self.ctx, self.n, self.m = h, ctx, n, m
        self.words = (m + 31) // 32
        self._keep = (row_ptr, col, labels) if d0 else None

    def set_edge_labels(self, edge_labels, validate: bool = False):
        """Edge label of every CSR entry (uint8 [m_dir], the same on both
        entries of an edge; ccpm_graph_set_edge_labels).  None removes them."""
        if edge_labels is None:
            self.ctx.check(lib.ccpm_graph_set_edge_labels(self.h, None, CCPM_HOST_PTRS), "ccpm_graph_set_edge_labels")
            self._el = None
            return
        check_edge_labels(edge_labels, self.m)
        p, dev = _ptr(edge_labels)
        flags = (CCPM_DEVICE_PTRS if dev else CCPM_HOST_PTRS) | (CCPM_VALIDATE if validate else 0)
        self.ctx.check(lib.ccpm_graph_set_edge_labels(self.h, p, flags), "ccpm_graph_set_edge_labels")
        self._el = edge_labels if dev else None     # borrowed device arrays must stay alive

    def close(self):
        if self.h:
            lib.ccpm_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check_edge_labels(edge_labels, m):
    """The library reads m bytes from the array it is given: one uint8 label
    per CSR entry, contiguous (ValueError otherwise)."""
    import torch
    if isinstance(edge_labels, torch.Tensor):
        ok_type = edge_labels.dtype == torch.uint8
        contiguous = edge_labels.is_contiguous()
    else:
        ok_type = isinstance(edge_labels, np.ndarray) and edge_labels.dtype == np.uint8
        contiguous = ok_type and edge_labels.flags["C_CONTIGUOUS"]
    if not ok_type:
        raise ValueError("edge labels must be a uint8 numpy array or tensor")
    if edge_labels.ndim != 1 or int(edge_labels.shape[0]) != m:
        raise ValueError(f"edge labels hold {int(edge_labels.shape[0])} entries, the graph {m}")
    if not contiguous:
        raise ValueError("edge labels must be contiguous")


def lcc_wide(ctx, graph, labels, edges, edge_labels=None, device_out=False):
    """LCC fixpoint for templates of up to 64 vertices with edge labels
    (ccpm_lcc_wide).  Returns (omega [n], edge bitmap [words], stats dict):
    host arrays (uint64, uint32), or with device_out CUDA tensors on the
    context's device (int64 and int32 holding the same bits)."""
    lab = np.ascontiguousarray(np.asarray(labels, dtype=np.uint8))
    ed = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    tel = None
    if edge_labels is not None:
        tel = np.ascontiguousarray(np.asarray(edge_labels, dtype=np.uint8))
        if tel.shape[0] != ed.shape[0] // 2:
            raise ValueError("one edge label per template edge")
    if device_out:
        import torch
        dev = f"cuda:{ctx.device}"
        omega = torch.empty(max(graph.n, 1), dtype=torch.int64, device=dev)
        bits = torch.empty(max(graph.words, 1), dtype=torch.int32, device=dev)
    else:
        omega = np.zeros(max(graph.n, 1), dtype=np.uint64)
        bits = np.zeros(max(graph.words, 1), dtype=np.uint32)
    st = WideStats()
    ctx.check(lib.ccpm_lcc_wide(ctx.h, graph.h, int(lab.shape[0]), _ptr(lab)[0], int(ed.shape[0] // 2),
                                _ptr(ed)[0], None if tel is None else _ptr(tel)[0], _ptr(omega)[0],
                                _ptr(bits)[0], 1 if device_out else 0, ctypes.byref(st)), "ccpm_lcc_wide")
    stats = {k: getattr(st, k) for k, _ in st._fields_}
    return omega[: graph.n], bits[: graph.words], stats


def batch_tuning(graph) -> dict:
    """The batch autotuner's choices for `graph` (ccpm_graph_batch_tuning)."""
    v = [ctypes.c_int(0) for _ in range(5)]
    ms = ctypes.c_double(0.0)
    lib.ccpm_graph_batch_tuning(graph.h, *[ctypes.byref(x) for x in v], ctypes.byref(ms))
    return {"workers": v[0].value, "grid_share": v[1].value, "search_split": v[2].value,
            "short_rows": v[3].value, "hub_degree": v[4].value, "slice_ms": ms.value}


class Template:
    def __init__(self, ctx, labels, edges):
        lab = np.ascontiguousarray(np.asarray(labels, dtype=np.uint8))
        ed = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
        h = ctypes.c_void_p()
        rc = lib.ccpm_tmpl_load(ctx.h if ctx else None, int(lab.shape[0]), _ptr(lab)[0],
                                int(ed.shape[0] // 2), _ptr(ed)[0], ctypes.byref(h))
        if rc:
            msg = lib.ccpm_last_error(ctx.h).decode() if ctx else "invalid template"
            raise CcpmError(rc, f"ccpm_tmpl_load: {msg}")
        self.h, self.ctx = h, ctx
        self.labels = [int(x) for x in lab]
        self.edges = [tuple(int(v) for v in e) for e in np.asarray(edges).reshape(-1, 2)]

    def generate(self, graph: Graph | None = None) -> int:
        n = ctypes.c_int()
        rc = lib.ccpm_constraints_generate(self.h, graph.h if graph else None, ctypes.byref(n))
        if rc:
            raise CcpmError(rc, "ccpm_constraints_generate")
        return n.value

    def describe(self, i: int) -> dict:
        info = ConstraintInfo()
        rc = lib.ccpm_constraints_describe(self.h, i, ctypes.byref(info))
        if rc:
            raise CcpmError(rc, "ccpm_constraints_describe")
        verts = [q for q in range(32) if (info.vert_mask >> q) & 1]
        heads = [q for q in range(32) if (info.head_mask >> q) & 1]
        edges = [[info.edges[k][0], info.edges[k][1]] for k in range(info.n_edges)]
        return {"kind": KIND_NAMES[info.kind], "verts": verts, "edges": edges, "heads": heads,
                "vert_mask": info.vert_mask, "head_mask": info.head_mask}

    def constraints(self):
        n = self.generate()
        return [self.describe(i) for i in range(n)]

    def set_order(self, order):
        o = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
        rc = lib.ccpm_tmpl_set_order(self.h, int(o.shape[0]), _ptr(o)[0])
        if rc:
            raise CcpmError(rc, "ccpm_tmpl_set_order")

    def close(self):
        if self.h:
            lib.ccpm_tmpl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Result:
    def __init__(self, graph: Graph, h):
        self.graph, self.h = graph, h

    def omega(self, out=None):
        if out is None:
            out = np.zeros(self.graph.n, dtype=np.uint32)
        p, dev = _ptr(out)
        self.graph.ctx.check(lib.ccpm_result_omega(self.h, p, self.graph.n, int(dev)), "ccpm_result_omega")
        return out

    def edge_bitmap(self, out=None):
        if out is None:
            out = np.zeros(self.graph.words, dtype=np.uint32)
        p, dev = _ptr(out)
        self.graph.ctx.check(lib.ccpm_result_edge_bitmap(self.h, p, self.graph.words, int(dev)),
                             "ccpm_result_edge_bitmap")
        return out

    def counts(self) -> dict:
        c = Counts()
        lib.ccpm_result_counts(self.h, ctypes.byref(c))
        return c.as_dict()

    def phase_rounds(self):
        c = self.counts()
        out = np.zeros(max(c["n_phases"], 1), dtype=np.int32)
        lib.ccpm_result_phase_rounds(self.h, _ptr(out)[0], int(c["n_phases"]))
        return [int(x) for x in out[: c["n_phases"]]]

    def logs(self):
        """Per-constraint log records, in the order the constraints ran."""
        out = []
        for i in range(max(self.counts()["n_phases"] - 1, 0)):
            rec = ConstraintLog()
            rc = lib.ccpm_result_constraint_log(self.h, i, ctypes.byref(rec))
            if rc:
                raise CcpmError(rc, "ccpm_result_constraint_log")
            out.append(rec.as_dict())
        return out

    def order(self):
        """Generated-order indices of the constraints, in the order they ran."""
        return [r["constraint"] for r in self.logs()]

    def matches(self, tmpl, list_cap: int = 0, vertex_counts: bool = False, entry_counts: bool = False,
                opts=None, device: bool = False):
        """ccpm_result_matches: (n_matches, list [min(n, list_cap), n0] int32,
        per-vertex counts uint64 [n] or None, per-entry counts uint64 [m] or
        None).  device=True returns CUDA tensors filled in place."""
        n0 = len(tmpl.labels)
        g = self.graph
        if device:
            import torch
            dev = torch.device("cuda", g.ctx.device)
            lst = torch.zeros((max(list_cap, 1), n0), dtype=torch.int32, device=dev)
            vc = torch.zeros(g.n, dtype=torch.int64, device=dev) if vertex_counts else None
            ec = torch.zeros(max(g.m, 1), dtype=torch.int64, device=dev) if entry_counts else None
        else:
            lst = np.zeros((max(list_cap, 1), n0), dtype=np.int32)
            vc = np.zeros(g.n, dtype=np.uint64) if vertex_counts else None
            ec = np.zeros(max(g.m, 1), dtype=np.uint64) if entry_counts else None
        nm = ctypes.c_uint64(0)
        p = lambda x: _ptr(x)[0] if x is not None else None
        rc = lib.ccpm_result_matches(g.ctx.h, self.h, tmpl.h, ctypes.byref(opts) if opts is not None else None,
                                     p(lst), int(list_cap), p(vc), p(ec), int(device), ctypes.byref(nm))
        g.ctx.check(rc, "ccpm_result_matches")
        k = min(int(nm.value), list_cap)
        return int(nm.value), lst[:k], vc, (ec[: g.m] if ec is not None else None)

    def export_state(self) -> bytes:
        """ccpm_state_export: the state as one self-describing byte blob."""
        n = ctypes.c_size_t(0)
        self.graph.ctx.check(lib.ccpm_state_export(self.h, None, ctypes.byref(n)), "ccpm_state_export")
        buf = ctypes.create_string_buffer(n.value)
        self.graph.ctx.check(lib.ccpm_state_export(self.h, buf, ctypes.byref(n)), "ccpm_state_export")
        return buf.raw[: n.value]

    def close(self):
        if self.h:
            lib.ccpm_result_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prune(ctx: Context, graph: Graph, tmpl: Template, opts: Options | None = None,
          result: Result | None = None, allow_budget: bool = False) -> Result:
    """ccpm_prune; reuses `result` when given."""
    h = ctypes.c_void_p(result.h.value if result is not None else None)
    rc = lib.ccpm_prune(ctx.h, graph.h, tmpl.h, ctypes.byref(opts) if opts is not None else None,
                        ctypes.byref(h))
    if rc and not (rc == CCPM_EBUDGET and allow_budget):
        if rc == CCPM_EBUDGET and h.value:
            Result(graph, h).close() if result is None else None
        ctx.check(rc, "ccpm_prune")
    if result is not None:
        return result
    return Result(graph, h)


def state_import(ctx: Context, graph: Graph, tmpl: Template, blob: bytes) -> Result:
    """ccpm_state_import: a result holding a saved state; prune it further with
    options(resume=1) and result=<this result>."""
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(bytes(blob), len(blob))
    ctx.check(lib.ccpm_state_import(ctx.h, graph.h, tmpl.h, buf, len(blob), ctypes.byref(h)), "ccpm_state_import")
    return Result(graph, h)


def lcc_fixpoint_noalloc(device, row_ptr, col, labels, tmpl_labels, tmpl_edges, omega, ebits, stream=None):
    """ccpm_lcc_fixpoint_noalloc: LCC to its fixpoint with no allocation inside
    the library, for callers that cannot allocate device memory while they
    run.  Graph arrays and the omega / ebits outputs are CUDA tensors the
    caller owns.  Returns (rounds, edges_scanned)."""
    import torch
    tl = np.ascontiguousarray(np.asarray(tmpl_labels, dtype=np.uint8))
    te = np.ascontiguousarray(np.asarray(tmpl_edges, dtype=np.int32).reshape(-1))
    arrays = {"row_ptr": row_ptr, "col": col, "labels": labels, "omega": omega, "ebits": ebits}
    for name, x in arrays.items():
        if not isinstance(x, torch.Tensor) or not x.is_contiguous():
            raise ValueError(f"{name} must be a contiguous torch tensor")
    n = int(row_ptr.numel()) - 1
    m = int(col.numel())
    want = {"row_ptr": ((torch.int64,), n + 1), "col": ((torch.int32,), m), "labels": ((torch.uint8,), n),
            "omega": ((torch.int32, torch.uint32), n), "ebits": ((torch.int32, torch.uint32), (m + 31) // 32)}
    for name, (dtypes, need) in want.items():
        x = arrays[name]
        if x.dtype not in dtypes:
            raise ValueError(f"{name} must have dtype {' or '.join(str(d) for d in dtypes)}, not {x.dtype}")
        if x.numel() < need:
            raise ValueError(f"{name} holds {x.numel()} elements, needs at least {need}")
    for name, x in arrays.items():
        if not x.is_cuda or x.device.index != int(device):
            raise ValueError(f"{name} must be a tensor on cuda:{int(device)}, not {x.device}")
    ptrs = [_ptr(x) for x in (row_ptr, col, labels, omega, ebits)]
    rounds = ctypes.c_int32()
    scanned = ctypes.c_int64()
    err = ctypes.create_string_buffer(256)
    rc = lib.ccpm_lcc_fixpoint_noalloc(int(device), ctypes.c_void_p(int(stream)) if stream else None,
                                       int(row_ptr.shape[0]) - 1, int(col.shape[0]),
                                       ptrs[0][0], ptrs[1][0], ptrs[2][0], int(tl.shape[0]), _ptr(tl)[0],
                                       int(te.shape[0] // 2), _ptr(te)[0], ptrs[3][0], ptrs[4][0],
                                       ctypes.byref(rounds), ctypes.byref(scanned), err, 256)
    if rc:
        raise CcpmError(rc, f"ccpm_lcc_fixpoint_noalloc: {err.value.decode()}")
    return rounds.value, scanned.value


def explore(ctx: Context, graph: Graph, base: Template, max_removed: int, opts: Options | None = None,
            allow_budget: bool = False, variants_cap: int = 4096):
    """ccpm_explore: (level found or -1, union Result, per-variant records,
    milliseconds spent building the candidate set)."""
    recs = (ExploreVariant * max(variants_cap, 1))()
    nv, lvl, msc = ctypes.c_int32(0), ctypes.c_int32(-1), ctypes.c_double(0.0)
    h = ctypes.c_void_p()
    rc = lib.ccpm_explore(ctx.h, graph.h, base.h, int(max_removed), ctypes.byref(opts) if opts is not None else None,
                          recs, int(variants_cap), ctypes.byref(nv), ctypes.byref(lvl), ctypes.byref(msc),
                          ctypes.byref(h))
    if rc and not (rc == CCPM_EBUDGET and allow_budget):
        ctx.check(rc, "ccpm_explore")
    out = [recs[i].as_dict() for i in range(min(nv.value, variants_cap))]
    return lvl.value, Result(graph, h), out, msc.value


def prune_batch(ctx: Context, graph: Graph, tmpls, opts: Options | None = None, results=None,
                allow_budget: bool = False):
    """ccpm_prune_batch over a list of Templates; reuses `results` when given."""
    T = len(tmpls)
    th = (ctypes.c_void_p * T)(*[t.h for t in tmpls])
    rh = (ctypes.c_void_p * T)(*[(r.h.value if r is not None else None) for r in (results or [None] * T)])
    rc = lib.ccpm_prune_batch(ctx.h, graph.h, T, th, ctypes.byref(opts) if opts is not None else None, rh)
    if rc and not (rc == CCPM_EBUDGET and allow_budget):
        ctx.check(rc, "ccpm_prune_batch")
    if results is not None:
        return results
    return [Result(graph, ctypes.c_void_p(rh[i])) for i in range(T)]


class Mlp:
    """The constraint-ordering network (BF16 tensor-core kernels in the library)."""

    def __init__(self, ctx: Context, seed: int = 1):
        h = ctypes.c_void_p()
        ctx.check(lib.ccpm_mlp_create(ctx.h, seed, ctypes.byref(h)), "ccpm_mlp_create")
        self.h, self.ctx = h, ctx

    def params(self) -> np.ndarray:
        out = np.zeros(MLP_PARAMS, dtype=np.float32)
        rc = lib.ccpm_mlp_get_params(self.h, _ptr(out)[0])
        if rc:
            raise CcpmError(rc, "ccpm_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        assert p.shape == (MLP_PARAMS,)
        rc = lib.ccpm_mlp_set_params(self.h, _ptr(p)[0])
        if rc:
            raise CcpmError(rc, "ccpm_mlp_set_params")

    def forward(self, x) -> np.ndarray:
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1, MLP_IN))
        y = np.zeros(x.shape[0], dtype=np.float32)
        rc = lib.ccpm_mlp_forward(self.h, x.shape[0], _ptr(x)[0], _ptr(y)[0])
        if rc:
            raise CcpmError(rc, "ccpm_mlp_forward")
        return y

    def gradient(self, x, t):
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1, MLP_IN))
        t = np.ascontiguousarray(np.asarray(t, dtype=np.float32).reshape(-1))
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        rc = lib.ccpm_mlp_gradient(self.h, x.shape[0], _ptr(x)[0], _ptr(t)[0], _ptr(g)[0], ctypes.byref(loss))
        if rc:
            raise CcpmError(rc, "ccpm_mlp_gradient")
        return g, loss.value

    def train(self, x, t, steps: int, batch: int = 256, lr: float = 1e-3, seed: int = 1) -> float:
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1, MLP_IN))
        t = np.ascontiguousarray(np.asarray(t, dtype=np.float32).reshape(-1))
        loss = ctypes.c_float()
        rc = lib.ccpm_mlp_train(self.h, x.shape[0], _ptr(x)[0], _ptr(t)[0], steps, batch, lr, seed,
                                ctypes.byref(loss))
        if rc:
            raise CcpmError(rc, "ccpm_mlp_train")
        return loss.value

    def close(self):
        if self.h:
            lib.ccpm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
