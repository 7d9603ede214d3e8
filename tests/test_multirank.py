"""The bench's reduction of the timed figures over ranks, on CPU with two gloo
ranks: the slowest rank's time, with the work summed over replicas (each rank
its own query) or taken once when the ranks shared one query (sources
sharded; the exchange itself is tested in test_shard.py)."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, edges = bench.reduce_over_ranks(100.0 + 50.0 * rank, 1_000_000 * (rank + 1), dist, "cpu")
    ms2, work = bench.reduce_over_ranks(100.0 + 50.0 * rank, 5_000_000, dist, "cpu", shared=True)
    out[rank] = (ms, edges, ms2, work)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_takes_slowest_time_and_all_arcs():
    world = 2
    with mp.get_context("spawn").Manager() as m:  # no fork of a threaded process
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        assert res[rank] == (150.0, 3_000_000.0, 150.0, 5_000_000.0)


def test_one_rank_is_unchanged():
    import bench

    assert bench.reduce_over_ranks(12.5, 7, None, "cpu") == (12.5, 7.0)
