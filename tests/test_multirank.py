"""Host logic of the N > 1 benchmark path (replicas only, no data exchange): two gloo ranks on
the CPU agree on the max-over-ranks timed region and the whole-job value."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [3.0, 5.0][rank]
    v = bench.whole_job_seconds(local, steps=4, world=world, dist=dist, device="cpu")
    out[rank] = v
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1] == pytest.approx(5.0 / (4 * 2))


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.whole_job_seconds(6.0, steps=3, world=1) == pytest.approx(2.0)
