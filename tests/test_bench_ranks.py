"""bench.py's multi-rank path (replicas only, no data-path collective): the
job time is the max over ranks.  Two gloo ranks on the CPU."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, e2e = bench.combine_ranks(10.0 + 5.0 * rank, 1.0 + rank, world, device="cpu")
    out[rank] = (ms, e2e)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_takes_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == (15.0, 2.0) and out[1] == (15.0, 2.0)


def test_combine_ranks_single_rank_is_identity():
    import bench
    assert bench.combine_ranks(3.0, 4.0, 1) == (3.0, 4.0)
