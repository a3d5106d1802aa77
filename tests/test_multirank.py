"""The multi-GPU path is replicas only: every rank runs the whole query on its
own GPU, and bench.py combines the ranks on the host (the slowest rank's time,
all ranks' units).  That host logic runs here on two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, times, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=ws)
    try:
        dist.barrier()
        t = bench.max_over_ranks(times[rank], ws, device="cpu")
        out[rank] = (t, bench.job_throughput(1000.0, t, ws))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(0.25, 0.5), (0.75, 0.125)])
def test_two_ranks_take_the_slowest_and_all_units(times):
    ws = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, _free_port(), list(times), out), nprocs=ws, join=True)
        res = dict(out)
    slowest = max(times)
    for rank in range(ws):
        t, value = res[rank]
        assert t == slowest                      # every rank sees the same, largest time
        assert value == ws * 1000.0 / slowest    # all ranks' units over that time


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5
    assert bench.job_throughput(1000.0, 0.5, 1) == 2000.0
