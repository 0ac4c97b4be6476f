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
    # a slowdown seen on one rank makes every rank measure again
    again = bench._any_rank(rank == 1, None)
    out[rank] = (t, u, again)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_sum_units():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (3.5, 4000.0, True) and out[1] == (3.5, 4000.0, True)


def test_single_process_is_identity():
    import bench
    assert bench.reduce_over_ranks(1.25, 10.0) == (1.25, 10.0)
    assert bench._any_rank(True) and not bench._any_rank(False)


def test_clock_records_that_are_measured_again():
    import bench
    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench._clocks_rejected(ok)
    assert not bench._clocks_rejected({**ok, "reasons": ["sw_power_cap"], "sm_mhz": 1800.0})
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench._clocks_rejected({**ok, "reasons": [r]})
    assert bench._clocks_rejected({**ok, "sm_mhz": 1200.0})        # stuck low, no reason
    assert not bench._clocks_rejected({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]})


def test_traffic_fingerprint_ignores_comments_only():
    """The DRAM traffic bench.py reports was captured on a given kernel source;
    its fingerprint ignores comments but not code."""
    import bench
    src = "// head\n__global__ void k(int *p) {\n    p[0] = 1;  /* one */\n}\n"
    same = "/* new text */\n__global__ void k(int *p) {   \n    p[0] = 1;  // one\n\n}\n"
    other = "__global__ void k(int *p) {\n    p[0] = 2;\n}\n"
    fp = lambda text: bench._sources_sha256(["x.cu"], read=lambda rel: text)
    assert fp(src) == fp(same) and fp(src) != fp(other)
