"""The N > 1 benchmark path is replicas only (independent problems per rank, no data-path
collective); its host logic -- the max of the per-rank times and the whole-job rate -- runs
here on two gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


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
    local_ms = [100.0, 150.0][rank]
    tmax, rate = bench.whole_job_rate(local_ms, 30.0, dist, None)
    out[rank] = (tmax, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_two_gloo_ranks():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        tmax, rate = out[r]
        assert tmax == 150.0                       # max over ranks
        assert abs(rate - 2 * 30.0 / 0.150) < 1e-9  # all ranks' units / the slowest rank's time


def test_whole_job_rate_single_process():
    import bench
    tmax, rate = bench.whole_job_rate(200.0, 30.0)
    assert tmax == 200.0 and abs(rate - 150.0) < 1e-12
