"""Learned ordering of non-local constraints: data, training and evaluation.

The plain pipeline (fixed order, Section 4.2) logs, for every constraint it
checks, the ordering features in the state where it was chosen, the omega bits
it removed (with its LCC re-run) and its device time.  The network learns
    target = -log2(1 + microseconds spent)
(optionally plus benefit_weight * log2(1 + bits removed)), i.e. how cheap the
constraint is to check in that state.  With CCPM_ORDER_LEARNED the pipeline
keeps the fixed order as a prior: a later constraint runs first only if it
is predicted more than twice as cheap as the fixed order's next one (the one
predicted cheapest among those), so that expensive checks wait for a state
that cheaper ones have already shrunk.  Every constraint is still checked, so
omega, the edge bitmap and the match count equal the fixed order's; only the
order, and with it the LCC round counts and the time, change.

Training and inference run in the library's BF16 tensor-core kernels; this
module only assembles arrays.
"""
from __future__ import annotations

import numpy as np

from . import ccpm


def target(rec, benefit_weight: float = 0.0) -> float:
    """log2(1 + bits removed) * benefit_weight - log2(1 + microseconds)."""
    removed = max(rec["bits_before"] - rec["bits_after"], 0)
    cost_us = 1000.0 * (rec["ms_search"] + rec["ms_lcc"])
    return float(benefit_weight * np.log2(1.0 + removed) - np.log2(1.0 + cost_us))


def collect_logs(ctx, graph, templates, repeats: int = 1, benefit_weight: float = 0.0, raw: bool = False):
    """Run the fixed-order pipeline on every template; return (X, y), or the
    raw log records when raw=True."""
    X, y, recs = [], [], []
    result = None
    for t in templates:
        h = t if isinstance(t, ccpm.Template) else ccpm.Template(ctx, t.labels, t.edges)
        for _ in range(repeats):
            result = ccpm.prune(ctx, graph, h, ccpm.options(), result=None, allow_budget=True)
            for rec in result.logs():
                recs.append(rec)
                X.append(rec["features"])
                y.append(target(rec, benefit_weight))
            result.close()
    if raw:
        return recs
    return np.asarray(X, dtype=np.float32).reshape(-1, ccpm.MLP_IN), np.asarray(y, dtype=np.float32)


def train(ctx, X, y, steps: int = 2000, batch: int = 256, lr: float = 2e-3, seed: int = 1):
    net = ccpm.Mlp(ctx, seed=seed)
    net.train(X, y, steps=steps, batch=batch, lr=lr, seed=seed)
    return net


def learned_options(net, **kw):
    o = ccpm.options(order_mode=ccpm.CCPM_ORDER_LEARNED, **kw)
    o.mlp = net.h.value
    return o


def targets_from(recs, benefit_weight: float = 0.0):
    X = np.asarray([r["features"] for r in recs], dtype=np.float32).reshape(-1, ccpm.MLP_IN)
    y = np.asarray([target(r, benefit_weight) for r in recs], dtype=np.float32)
    return X, y


def choose(ctx, graph, templates, net, max_embeddings=1 << 32, repeats: int = 1):
    """The fixed order decides whether the learned one is used: both prune the same templates
    one at a time (the learned options also run a warm-up pass); the learned
    order is kept only if its total device time is lower.  Returns
    (use_learned, ms_fixed, ms_learned).  Outputs are identical either way;
    only the order, and so the time, differs."""
    fixed = ccpm.options(max_embeddings=max_embeddings)
    learned = learned_options(net, max_embeddings=max_embeddings)
    hs = [t if isinstance(t, ccpm.Template) else ccpm.Template(ctx, t.labels, t.edges) for t in templates]
    totals = []
    for o in (fixed, learned):
        res = [None] * len(hs)
        for i, h in enumerate(hs):                       # warm-up
            res[i] = ccpm.prune(ctx, graph, h, o, result=res[i], allow_budget=True)
        ms = 0.0
        for _ in range(repeats):
            for i, h in enumerate(hs):
                res[i] = ccpm.prune(ctx, graph, h, o, result=res[i], allow_budget=True)
                ms += res[i].counts()["ms_total"]
        totals.append(ms)
        for r in res:
            r.close()
    return totals[1] < totals[0], totals[0], totals[1]
