"""The multi-rank host logic (instance sharding, barrier, maximum of per-rank times, sum of work)
with two gloo ranks on the CPU."""
import os
import socket

import pytest

from paper_1902_10432_gb300 import ranks


def test_shard_round_robin_covers_each_instance_once():
    for n in (0, 1, 5, 64):
        for world in (1, 2, 3, 8):
            got = sorted(i for r in range(world) for i in ranks.shard(n, r, world))
            assert got == list(range(n))
            sizes = [len(ranks.shard(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        ranks.shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    r = ranks.Ranks(backend="gloo")
    mine = ranks.shard(64, r.rank, r.world)
    cells = sum(1000 + i for i in mine)  # per-instance work of uneven size
    r.barrier()
    t_max = r.max(1.5 + r.rank)  # rank-dependent "times"
    total = r.sum(cells)
    out[rank] = (r.root, mine, t_max, total)
    r.close()


def test_two_gloo_ranks_time_with_max_and_add_the_work():
    import torch.multiprocessing as mp

    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert res[0][0] and not res[1][0]  # only rank 0 reports
    assert sorted(res[0][1] + res[1][1]) == list(range(64))
    for rank in range(world):
        assert res[rank][2] == 1.5 + (world - 1)  # the slowest rank's time
        assert res[rank][3] == sum(1000 + i for i in range(64))  # every instance counted once
