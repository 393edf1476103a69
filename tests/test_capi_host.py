"""C-ABI checks that need no GPU: the library loads, exports every function
include/ccpm.h declares, validates templates, and its C++ constraint
generation (Table 3, Alg. 2) equals the oracle's, constraint by constraint."""
import json
import os
import re

import numpy as np
import pytest

from paper_1912_08453_gb300 import ccpm
from paper_1912_08453_gb300 import workloads as wl
from oracle import constraints as cgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ccpm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ccpm_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_function():
    names = declared_functions()
    assert len(names) >= 19
    for name in names:
        assert hasattr(ccpm.lib, name), name
    assert sorted(ccpm.EXPORTED) == names


def test_template_validation():
    with pytest.raises(ccpm.CcpmError):
        ccpm.Template(None, [0, 1, 2, 3], [(0, 1), (2, 3)])          # disconnected
    with pytest.raises(ccpm.CcpmError):
        ccpm.Template(None, [0], [])                                   # n0 < 2
    with pytest.raises(ccpm.CcpmError):
        ccpm.Template(None, [0, 1], [(0, 0)])                          # self loop
    with pytest.raises(ccpm.CcpmError):
        ccpm.Template(None, [0, 1], [(0, 1), (1, 0)])                  # duplicate
    with pytest.raises(ccpm.CcpmError):
        ccpm.Template(None, list(range(33)), [(i, i + 1) for i in range(32)])   # n0 > 32


def product_constraints(labels, edges):
    t = ccpm.Template(None, labels, edges)
    return t.constraints()


def oracle_constraints(labels, edges):
    return [{"kind": cgen.KIND_NAMES[c.kind], "verts": sorted(c.verts),
             "edges": sorted([list(e) for e in c.edges]), "heads": sorted(c.heads)}
            for c in cgen.generate(labels, edges)]


def strip(cs):
    return [{k: c[k] for k in ("kind", "verts", "edges", "heads")} for c in cs]


def test_golden_constraint_sets():
    fx = json.load(open(os.path.join(ROOT, "tests", "golden", "constraint_generation.json")))
    for case in fx["cases"]:
        got = strip(product_constraints(case["labels"], case["edges"]))
        assert got == case["expect"], case["name"]


@pytest.mark.parametrize("seed", range(60))
def test_constraints_equal_oracle(seed):
    rng = np.random.default_rng(seed)
    n0 = int(rng.integers(3, 10))
    extra = int(rng.integers(0, 4))
    n_labels = int(rng.integers(1, 5))
    t = wl.random_template(seed, n0, extra, list(range(n_labels)))
    assert strip(product_constraints(t.labels, t.edges)) == oracle_constraints(t.labels, t.edges)


def test_explicit_order_permutes():
    t = ccpm.Template(None, [0, 1, 2, 3], [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])
    base = t.constraints()
    perm = list(reversed(range(len(base))))
    t.set_order(perm)
    got = [t.describe(i) for i in range(len(base))]
    assert got == [base[j] for j in perm]
    with pytest.raises(ccpm.CcpmError):
        t.set_order([0] * len(base))
