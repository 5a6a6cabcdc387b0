"""Sharding of independent circuits across ranks (host logic, no GPU): the
greedy partition's invariants, a worked example, its balance on the batched
workload, and a two-rank gloo run in which each rank computes its share and
the gathered results equal the serial ones."""
import os
import socket

import numpy as np
import pytest

from paper_2511_19291_gb300 import shard as SH
from paper_2511_19291_gb300 import workloads as W


def _check_partition(costs, world, parts):
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))          # every circuit, once
    assert all(p == sorted(p) for p in parts)
    loads = [sum(costs[i] for i in p) for p in parts]
    if costs:
        # list scheduling: the largest load is at most the mean plus the largest cost
        assert max(loads) <= sum(costs) / world + max(costs)
    return loads


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_partition_invariants(world, seed):
    rng = W.SplitMix64(900 + seed)
    costs = [SH.circuit_cost(rng.randint(3, 20), rng.randint(0, 300)) for _ in range(57)]
    parts = SH.partition(costs, world)
    assert len(parts) == world
    _check_partition(costs, world, parts)
    assert parts == SH.partition(list(costs), world)  # the same on every rank
    for r in range(world):
        assert SH.shard(costs, world, r) == parts[r]


def test_partition_worked_example():
    # longest first, each to the least-loaded rank (ties to the lower rank):
    # 7 -> 0; 5 -> 1; 4 -> 1 (9); 3 -> 0 (10); 3 -> 1 (12); 2 -> 0 (12)
    assert SH.partition([7, 5, 4, 3, 3, 2], 2) == [[0, 3, 5], [1, 2, 4]]
    assert SH.partition([3, 3, 3], 3) == [[0], [1], [2]]
    assert SH.partition([], 4) == [[], [], [], []]
    assert SH.partition([5], 3) == [[0], [], []]


def test_partition_rejects_bad_input():
    with pytest.raises(ValueError):
        SH.partition([1, 2], 0)
    with pytest.raises(ValueError):
        SH.partition([1, -2], 2)
    with pytest.raises(ValueError):
        SH.shard([1, 2], 2, 2)
    with pytest.raises(ValueError):
        SH.circuit_cost(-1, 3)


def test_batched_workload_balance():
    """The 512-circuit workload over 2, 4 and 8 ranks: within 2 % of the mean
    load (its largest circuits are small against a rank's share)."""
    wl = W.batched_workload(count=512)
    costs = SH.workload_costs(wl)
    for world in (2, 4, 8):
        loads = _check_partition(costs, world, SH.partition(costs, world))
        assert max(loads) / (sum(loads) / world) < 1.02, (world, loads)


# ------------------------------------------------------------ two gloo ranks
def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _small_batch():
    return W.batched_workload(count=10, wmin=3, wmax=6, dmin=1, dmax=3, config_index=11)


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
        wl = _small_batch()
        mine = SH.shard(SH.workload_costs(wl), world, rank)
        res = {}
        for i in mine:
            w = wl[i]
            e, g = oracle.grad_stored(w.circuit, w.params, w.terms)
            res[i] = (float(e), np.asarray(g, dtype=float).tolist())
        got = [None] * world
        dist.all_gather_object(got, res)  # gathering results, not a data-path exchange
        dist.destroy_process_group()
        q.put((rank, got))
    except Exception as exc:  # reported to the parent test
        q.put((rank, repr(exc)))


def test_two_gloo_ranks_shard_the_batch():
    import multiprocessing as mp

    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = _small_batch()
    parts = SH.partition(SH.workload_costs(wl), 2)
    for r in range(2):
        assert not isinstance(out[r], str), out[r]
        got = out[r]
        # each rank computed exactly its share; both see the same gathered list
        assert [sorted(d) for d in got] == parts
        assert got == out[0]
    merged = {i: v for d in out[0] for i, v in d.items()}
    assert sorted(merged) == list(range(len(wl)))
    for i, w in enumerate(wl):
        e, g = oracle.grad_stored(w.circuit, w.params, w.terms)
        assert merged[i][0] == float(e)
        np.testing.assert_array_equal(np.asarray(merged[i][1]), np.asarray(g, dtype=float))
