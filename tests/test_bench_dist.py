"""The N > 1 bench path on CPU: replicas on two gloo ranks, the slowest rank's
time and the whole-job throughput (no GPU, no data-path collective)."""
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


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, world)  # rank 1 is slower
    v = bench.whole_job_value(1000, 4, world, t)
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_max_time_and_value():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    for rank in (0, 1):
        t, v = out[rank]
        assert t == 15.0
        assert v == pytest.approx(1000 * 4 * 2 / 0.015)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_value(10, 2, 1, 4.0) == pytest.approx(5000.0)
