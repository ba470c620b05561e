"""The N > 1 bench path on the CPU: two gloo ranks agree on the slowest rank's time.

With several GPUs every rank computes its own determinant (independent
problems, weak scaling) and the bench reports work of all ranks over the
slowest rank's time; no collective touches the data path.
"""
import os
import socket

import pytest
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local = 10.0 + 5.0 * rank
    results[rank] = bench.max_over_ranks(local, device="cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = tmp.get_context("spawn")
    manager = ctx.Manager()
    results = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert results[0] == results[1] == 15.0


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
