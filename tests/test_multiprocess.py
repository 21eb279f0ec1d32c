"""The multi-process (replicas) path of the benchmark on CPU: two gloo ranks
shard the sweep's frames without overlap, agree on the slowest rank's time
and report the whole-job rate; the reference arm does no work off rank 0."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        frames = bench.frames_list()
        mine = bench.shard_frames(frames, rank, world)
        shards = [None] * world
        dist.all_gather_object(shards, mine)
        slow = bench.max_over_ranks(1.0 + rank)
        rate = bench.whole_job_rate(len(mine), world, slow)
        out.put((rank, shards, slow, rate, len(frames)))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, shards, slow, rate, n in res:
        flat = [f for s in shards for f in s]
        assert len(flat) == n and len(set(flat)) == n          # disjoint and complete
        assert slow == 2.0                                      # the slowest rank's time on every rank
        assert rate == pytest.approx(len(shards[rank]) * world / 2.0)


def test_reference_arm_idle_off_rank0(monkeypatch):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(steps=2, warmup=1, gpus=2)
    assert bench.run_reference(args) is None
