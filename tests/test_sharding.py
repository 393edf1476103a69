"""Host logic of running on several ranks: dealing independent templates to
ranks and reducing the step over ranks, with world_size-2 gloo process groups
on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1912_08453_gb300.sharding import deal, reduce_step


def test_deal_covers_every_problem_once():
    costs = [5, 1, 9, 3, 3, 7, 2, 8, 6, 4]
    for world in (1, 2, 3, 4, 16):
        share = deal(costs, world)
        assert len(share) == world
        flat = sorted(i for s in share for i in s)
        assert flat == list(range(len(costs)))
        assert all(s == sorted(s) for s in share)


def test_deal_is_balanced_and_deterministic():
    costs = [float((7 * i) % 11 + 1) for i in range(64)]
    for world in (2, 4, 8):
        share = deal(costs, world)
        loads = [sum(costs[i] for i in s) for s in share]
        # longest-first greedy: the most loaded rank exceeds the mean by at most one problem
        assert max(loads) <= sum(costs) / world + max(costs)
        assert share == deal(costs, world)


def test_deal_single_rank_and_ties():
    assert deal([1, 1, 1], 1) == [[0, 1, 2]]
    assert deal([1, 1, 1, 1], 2) == [[0, 2], [1, 3]]
    assert deal([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        deal([1], 0)


def test_reduce_without_process_group_is_local():
    assert reduce_step(3.5, 10, True) == (3.5, 10.0, True)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank prunes its share of 10 templates; the step time is its
        # own, the units its own; ok is False on rank 1 only
        costs = [5, 1, 9, 3, 3, 7, 2, 8, 6, 4]
        share = deal(costs, world)[rank]
        ms = sum(costs[i] for i in share)
        units = 100 * len(share)
        out[rank] = reduce_step(ms, units, ok=(rank != 1))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_reduce_step_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    costs = [5, 1, 9, 3, 3, 7, 2, 8, 6, 4]
    loads = [sum(costs[i] for i in s) for s in deal(costs, world)]
    for r in range(world):
        ms, units, ok = out[r]
        assert ms == max(loads)
        assert units == 100 * len(costs)
        assert ok is False
