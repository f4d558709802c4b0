"""The N > 1 bench path on CPU: two gloo ranks, each timing its own replica,
reduce to the slowest rank's time and the summed work (weak scaling), and
each rank's replica draws different random streams."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.reduce_over_ranks(100.0 + 50.0 * rank, 1000 * (rank + 1))
    from oracle import philox
    seed = 1 + 1000 * rank                       # bench's per-rank replica seed
    p = philox.momentum(seed, 0, 4, 3)
    gathered = [torch.zeros(4, 3, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, torch.tensor(p))
    out[rank] = (ms, units, [g.numpy().tolist() for g in gathered])
    dist.destroy_process_group()


def test_two_rank_reduction_and_independent_replicas():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        ms, units, streams = out[r]
        assert ms == 150.0
        assert units == 3000.0
        assert streams[0] != streams[1]


def test_single_process_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks(12.5, 7) == (12.5, 7)
