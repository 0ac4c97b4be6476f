"""The N > 1 path of bench.py: independent replicas, one process per GPU.
The whole-job figure is the units of every rank over the slowest rank's time.
Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [2.0, 3.5][rank]
    units = [1000.0, 3000.0][rank]
    t, u = bench.reduce_over_ranks(seconds, units, None)
    out[rank] = (t, u)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_sum_units():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (3.5, 4000.0) and out[1] == (3.5, 4000.0)


def test_single_process_is_identity():
    import bench
    assert bench.reduce_over_ranks(1.25, 10.0) == (1.25, 10.0)
