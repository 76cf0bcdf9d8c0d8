"""The N > 1 host path on CPU: two gloo ranks run the benchmark's control
plane (barrier, max over ranks) and the solve partition, with no GPU."""
import os
import socket

import pytest

from paper_0901_1053_gb300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    from paper_0901_1053_gb300 import workloads as wl
    d = bench.Dist(world)
    d.barrier()
    mx = d.max(10.0 + rank)
    solves = wl.batch_solves(count=9, seed=5, n_lo=8, n_hi=24)
    mine = [w.name for w in sharding.shard_workloads(solves, world, rank)]
    d.barrier()
    d.close()
    q.put((rank, mx, mine))


def test_two_gloo_ranks_agree_on_max_and_partition():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [11.0, 11.0]
    names0, names1 = set(res[0][2]), set(res[1][2])
    assert not names0 & names1
    assert len(names0 | names1) == 9


def test_partition_is_balanced_and_deterministic():
    costs = [9, 1, 8, 2, 7, 3, 6, 4, 5]
    a = sharding.shard_by_cost(costs, 3)
    assert a == sharding.shard_by_cost(costs, 3)
    loads = [sum(costs[i] for i in part) for part in a]
    assert max(loads) <= 4.0 / 3.0 * sum(costs) / 3 + 1e-9   # LPT bound
    assert max(loads) - min(loads) <= max(costs)
    assert sorted(i for part in a for i in part) == list(range(9))
    assert sharding.shard_by_cost(costs, 1) == [list(range(9))]
    with pytest.raises(ValueError):
        sharding.shard_by_cost(costs, 0)
