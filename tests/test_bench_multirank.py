"""The bench's multi-rank host logic on CPU: two gloo ranks reduce a timed
region to the slowest rank's time and the summed agent-updates (the whole-job
figure rank 0 prints), and the reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed 10 + r ms over 1000 * (r + 1) agent-updates
        ms, upd = bench.reduce_over_ranks(10.0 + rank, 1000 * (rank + 1), dist, "cpu")
        out[rank] = (ms, upd)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_slowest_time_and_summed_updates():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (11.0, 3000.0)


def test_no_process_group_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(7.5, 123, None, "cpu") == (7.5, 123)


def test_reference_arm_works_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        sample, steps, warmup, gpus, n = 0, 1, 1, 2, 10_000_000
        workload, sort_every, presort = "blobs", 10, False

    assert bench.run_reference(Args, 1, 2) == 0
    assert capsys.readouterr().out == ""
