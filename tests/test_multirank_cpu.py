"""The multi-rank host logic of the benchmark, on CPU with the gloo backend and
two ranks: independent systems are split over ranks by their n^3 cost with no
data-path collective; only timings (max), counts (sum) and latency lists
(gathered) cross ranks, and every rank agrees on the split."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, costs, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        parts = bench.shard_balanced(costs, world)
        mine = parts[rank]
        t_local = 1.0 + rank  # this rank's "time"
        conv_local = float(len(mine))
        t_max = bench.reduce_over_ranks([t_local], "max")[0]
        conv_all = bench.reduce_over_ranks([conv_local], "sum")[0]
        lat = bench.gather_lists([10.0 * rank + k for k in range(3)])
        out.put((rank, parts, t_max, conv_all, lat, bench.dist_env()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_and_reduce():
    world = 2
    costs = [float(n) ** 3 for n in (16, 256, 40, 200, 128, 130, 64, 250, 17, 90, 180, 33)]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, costs, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts0, parts1 = got[0][1], got[1][1]
    assert parts0 == parts1  # every rank computes the same split
    flat = sorted(parts0[0] + parts0[1])
    assert flat == list(range(len(costs)))  # disjoint and complete
    loads = [sum(costs[i] for i in q) for q in parts0]
    assert max(loads) <= 0.6 * sum(costs)  # balanced by cost
    for rank, _, t_max, conv_all, lat, env in got:
        assert t_max == 2.0
        assert conv_all == float(len(costs))
        assert sorted(lat) == [0.0, 1.0, 2.0, 10.0, 11.0, 12.0]
        assert env == (world, rank, rank)


def test_shard_balanced_single_rank_and_determinism():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    costs = [5.0, 1.0, 5.0, 3.0]
    assert bench.shard_balanced(costs, 1) == [[0, 1, 2, 3]]
    assert bench.shard_balanced(costs, 2) == bench.shard_balanced(list(costs), 2)
    assert bench.reduce_over_ranks([1.0, 2.0], "max") == [1.0, 2.0]  # no process group: identity
