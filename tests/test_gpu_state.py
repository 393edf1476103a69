"""Checkpoint/resume through the C ABI: ccpm_state_export / ccpm_state_import
and ccpm_prune with options.resume.

Pruning only removes candidates that no match uses (Section 4), so a saved
state of the same graph and template contains every match and a prune resumed
from it must end in the same omega*, E* and match count as a fresh run (and as
the oracle).
"""
import struct

import numpy as np
import pytest

from paper_1912_08453_gb300 import workloads as wl
from oracle import pipeline

pytestmark = pytest.mark.gpu

# a tree plus one triangle, and a 4-cycle with a pendant path (both need NLCC)
TREETRI6 = ([5, 4, 8, 7, 4, 5], [(0, 1), (1, 2), (1, 3), (3, 4), (3, 5), (2, 3)])
C4P6 = ([7, 8, 7, 4, 4, 6], [(0, 1), (1, 2), (2, 3), (3, 0), (0, 4), (4, 5)])


@pytest.fixture(scope="module")
def env():
    from paper_1912_08453_gb300 import ccpm
    ctx = ccpm.Context(0)
    g = wl.rmat_graph(16, labels="degree")
    graph = ccpm.Graph(ctx, g.row_ptr, g.col, g.labels)
    yield ccpm, ctx, g, graph
    graph.close()
    ctx.close()


def snapshot(r):
    return dict(omega=r.omega(), ebits=r.edge_bitmap(), counts=r.counts(), phases=r.phase_rounds())


@pytest.mark.parametrize("tmpl", [TREETRI6, C4P6], ids=["treetri6", "c4p6"])
def test_round_trip(env, tmpl):
    ccpm, ctx, g, graph = env
    t = ccpm.Template(ctx, *tmpl)
    r = ccpm.prune(ctx, graph, t, ccpm.options())
    blob = r.export_state()
    r2 = ccpm.state_import(ctx, graph, t, blob)
    a, b = snapshot(r), snapshot(r2)
    np.testing.assert_array_equal(a["omega"], b["omega"])
    np.testing.assert_array_equal(a["ebits"], b["ebits"])
    assert a["counts"] == b["counts"] and a["phases"] == b["phases"]
    assert r2.export_state() == blob
    r.close(); r2.close(); t.close()


@pytest.mark.parametrize("tmpl", [TREETRI6, C4P6], ids=["treetri6", "c4p6"])
def test_resume_after_checkpoint(env, tmpl):
    """Stop before the final search, save, load, finish: identical to one run
    and to the oracle."""
    ccpm, ctx, g, graph = env
    t = ccpm.Template(ctx, *tmpl)
    full = snapshot(ccpm.prune(ctx, graph, t, ccpm.options()))
    part = ccpm.prune(ctx, graph, t, ccpm.options(run_final=0))
    blob = part.export_state()
    part.close()
    r = ccpm.state_import(ctx, graph, t, blob)
    ccpm.prune(ctx, graph, t, ccpm.options(resume=1), result=r)
    got = snapshot(r)
    ref = pipeline.run(g.row_ptr, g.col, g.labels, *tmpl)
    for s in (full, got):
        np.testing.assert_array_equal(s["omega"], ref.omega)
        np.testing.assert_array_equal(s["ebits"], ref.ebits)
        assert s["counts"]["match_embeddings"] == ref.match_embeddings
        assert s["counts"]["count_valid"] == int(ref.count_valid)
    assert ref.match_embeddings > 0
    # resuming from the finished state changes nothing either
    ccpm.prune(ctx, graph, t, ccpm.options(resume=1), result=r)
    again = snapshot(r)
    np.testing.assert_array_equal(again["omega"], ref.omega)
    np.testing.assert_array_equal(again["ebits"], ref.ebits)
    assert again["counts"]["match_embeddings"] == ref.match_embeddings
    r.close(); t.close()


HEADER = struct.Struct("<8sIIqqqQQIIQQ16x")     # the 96-byte header ccpm.h describes


def fnv1a(data: bytes) -> int:
    h = 0xcbf29ce484222325
    for b in data:
        h = ((h ^ b) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def test_resume_from_lcc_fixpoint_blob(env):
    """A blob written by hand from the documented layout, holding the state
    after the initial LCC alone (from the allocation-free LCC entry point):
    resuming from it finishes the non-local constraints and the final search
    with the oracle's answer."""
    import torch
    ccpm, ctx, g, graph = env
    tl, te = C4P6
    t = ccpm.Template(ctx, tl, te)
    r = ccpm.prune(ctx, graph, t, ccpm.options())
    blob = r.export_state()
    r.close()
    (magic, version, hbytes, n, m, words, gfp, tfp, cbytes, nph, pbytes, pfnv) = HEADER.unpack_from(blob)
    assert magic == b"CCPMSTAT" and hbytes == HEADER.size == 96 and n == g.n and m == g.m_dir
    assert words == (m + 31) // 32 and pbytes == len(blob) - 96 and pfnv == fnv1a(blob[96:])
    dev = torch.device("cuda", 0)
    om = torch.zeros(n, dtype=torch.int32, device=dev)
    eb = torch.zeros(words + 1, dtype=torch.int32, device=dev)
    ccpm.lcc_fixpoint_noalloc(0, torch.as_tensor(g.row_ptr, device=dev), torch.as_tensor(g.col, device=dev),
                              torch.as_tensor(g.labels, device=dev), tl, te, om, eb)
    torch.cuda.synchronize()
    off = 96 + cbytes + 4 * nph
    payload = bytearray(blob[96:])
    payload[off - 96: off - 96 + 4 * n] = om.cpu().numpy().view(np.uint32).tobytes()
    payload[off - 96 + 4 * n:] = eb[:words].cpu().numpy().view(np.uint32).tobytes()
    head = HEADER.pack(magic, version, hbytes, n, m, words, gfp, tfp, cbytes, nph, pbytes, fnv1a(bytes(payload)))
    r = ccpm.state_import(ctx, graph, t, head + bytes(payload))
    np.testing.assert_array_equal(r.omega(), om.cpu().numpy().view(np.uint32))
    ccpm.prune(ctx, graph, t, ccpm.options(resume=1), result=r)
    ref = pipeline.run(g.row_ptr, g.col, g.labels, tl, te)
    got = snapshot(r)
    np.testing.assert_array_equal(got["omega"], ref.omega)
    np.testing.assert_array_equal(got["ebits"], ref.ebits)
    assert got["counts"]["match_embeddings"] == ref.match_embeddings
    r.close(); t.close()


def test_import_rejects_bad_blobs(env):
    ccpm, ctx, g, graph = env
    t = ccpm.Template(ctx, *TREETRI6)
    r = ccpm.prune(ctx, graph, t, ccpm.options())
    blob = r.export_state()
    r.close()
    other = ccpm.Template(ctx, *C4P6)
    with pytest.raises(ccpm.CcpmError) as e:
        ccpm.state_import(ctx, graph, other, blob)
    assert e.value.code == ccpm.CCPM_EINVAL
    for bad in (blob[:50], blob[:-4], b"X" + blob[1:],
                blob[:200] + bytes([blob[200] ^ 1]) + blob[201:]):
        with pytest.raises(ccpm.CcpmError) as e:
            ccpm.state_import(ctx, graph, t, bad)
        assert e.value.code == ccpm.CCPM_EINVAL
    g2 = wl.rmat_graph(12, labels="degree")
    graph2 = ccpm.Graph(ctx, g2.row_ptr, g2.col, g2.labels)
    with pytest.raises(ccpm.CcpmError):
        ccpm.state_import(ctx, graph2, t, blob)
    graph2.close()
    # resume needs a state of this template
    with pytest.raises(ccpm.CcpmError):
        ccpm.prune(ctx, graph, t, ccpm.options(resume=1))
    r_other = ccpm.prune(ctx, graph, other, ccpm.options())
    with pytest.raises(ccpm.CcpmError):
        ccpm.prune(ctx, graph, t, ccpm.options(resume=1), result=r_other)
    r_other.close(); other.close(); t.close()
