"""Multi-GPU runs are replicas (the path has no exchange step as
configured): every rank solves its own copy and the job's time is the
slowest rank's.  This covers that host-side logic with world_size 2 on the
gloo backend (CPU), as the benchmark's torchrun launch uses it."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 1 + r seconds and its e2e 10 - r seconds
    vals = bench.max_over_ranks([1.0 + rank, 10.0 - rank], dist)
    out[rank] = torch.tensor(vals)
    # the whole-job value: solves of all ranks over the slowest rank's time
    steps = 5
    value = world * steps / vals[0]
    out[world + rank] = torch.tensor([value, 0.0])
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r].tolist() == [2.0, 10.0]          # max over the two ranks
        assert out[world + r][0].item() == pytest.approx(world * 5 / 2.0)


def test_max_over_ranks_single_process_is_identity():
    import bench
    assert bench.max_over_ranks([3.0, 4.0], None) == [3.0, 4.0]
