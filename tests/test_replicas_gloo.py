"""The multi-GPU path is replicas only (one view per rank, no collective on
the data path): the bench's cross-rank timing (max over ranks) and the
whole-job throughput, run as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r took 4 + r ms per step: the job's time is the slowest rank's
    ms = bench.max_over_ranks(4.0 + rank, torch.device("cpu"), world)
    mpix = bench.whole_job_mpix(1280 * 720, ms, world)
    out[rank] = (ms, mpix)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        ms, mpix = out[r]
        assert ms == 5.0
        assert mpix == pytest.approx(2 * 1280 * 720 / 5e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    import torch
    import bench
    assert bench.max_over_ranks(4.5, torch.device("cpu"), 1) == 4.5
    assert bench.whole_job_mpix(921600, 4.5, 1) == pytest.approx(921600 / 4.5e-3 / 1e6)
