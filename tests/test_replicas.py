"""Host logic of the multi-GPU layout (replicas of independent problems), run as
two gloo ranks on the CPU: problem sharding, per-rank seeds, and the whole-job
throughput taken over the slowest rank."""
import os
import socket

import pytest

from paper_1009_0881_gb300 import replicas


def test_shard_is_a_balanced_partition():
    for count in (0, 1, 7, 64, 65):
        for world in (1, 2, 3, 8):
            parts = [replicas.shard(count, r, world) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(count))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def test_replica_seeds_distinct():
    assert len({replicas.replica_seed(r) for r in range(8)}) == 8


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed 100 units in (r + 1) * 10 ms
        value, slowest = replicas.aggregate_throughput(100.0, (rank + 1) * 10.0, world)
        mine = replicas.shard(64, rank, world)
        out[rank] = (value, slowest, mine)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in (0, 1):
        value, slowest, _ = res[rank]
        assert slowest == 20.0
        assert value == pytest.approx(2 * 100.0 / 0.020)
    assert sorted(res[0][2] + res[1][2]) == list(range(64))


def test_single_process_identity():
    value, slowest = replicas.aggregate_throughput(50.0, 5.0, 1)
    assert slowest == 5.0 and value == pytest.approx(50.0 / 0.005)
