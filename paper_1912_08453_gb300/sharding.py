"""Independent pruning problems over several ranks, one GPU each.

Templates pruned over the same resident graph share nothing but the graph: it
is replicated on every rank and the templates are dealt to the ranks, each of
which prunes its share with no exchange on the data path.  The only
collectives reduce the step time (maximum over ranks: the job is done when the
slowest rank is) and the work done (sum over ranks).  A single template does
not shard here; several ranks then run independent replicas of it.
"""
from __future__ import annotations


def deal(costs, world: int):
    """Longest-processing-time-first assignment of problems to ranks.

    costs[i] is the predicted cost of problem i (e.g. its time in a warm-up
    run).  Problems are taken in decreasing cost (ties: lower index first) and
    each goes to the currently least loaded rank (ties: lower rank).  Returns
    one list of problem indices per rank, each in increasing index order.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    share = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        share[r].append(i)
        load[r] += float(costs[i])
    return [sorted(s) for s in share]


def reduce_step(ms: float, units: float, ok: bool = True, device=None):
    """(max of ms, sum of units, all ok) over the ranks of the default
    process group; the local values when torch.distributed is not running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units), bool(ok)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    f = torch.tensor([1 if ok else 0], dtype=torch.int32, device=device)
    dist.all_reduce(f, op=dist.ReduceOp.MIN)
    return float(t[0].item()), float(u.item()), bool(f.item())
