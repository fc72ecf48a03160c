"""The N > 1 path on CPU: two gloo ranks run the cross-rank pieces of the
bench (the barrier + maximum of the timed region, the whole-job MLUPS, and
the round-robin shard of the batched sweep's runs), which is all the ranks
share; the data path itself has no collective."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 0.5 + rank  # this rank's timed seconds
        slowest = bench._slowest_rank_seconds(local, world, torch.device("cpu"))
        shard = bench._batch_shard(64, rank, world)
        q.put((rank, slowest, shard))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_ranks_agree_on_slowest_time_and_shard_runs(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    # every rank sees the slowest rank's time
    assert all(s == 0.5 + (world - 1) for _, s, _ in out)
    # the shards are disjoint and cover all runs
    runs = sorted(i for _, _, sh in out for i in sh)
    assert runs == list(range(64))
    assert all(len(sh) == 64 // world for _, _, sh in out)


def test_whole_job_mlups():
    # two ranks of 1000 nodes, 10 steps each, the slowest 1.5 s
    assert bench._aggregate_mlups(1000, 10, 2, 1.5) == pytest.approx(1000 * 10 * 2 / 1.5 / 1e6)
    assert bench._slowest_rank_seconds(0.25, 1, None) == 0.25
    assert bench._batch_shard(5, 0, 1) == [0, 1, 2, 3, 4]
