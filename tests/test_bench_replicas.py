"""The benchmark's multi-GPU mode runs one independent replica per rank (the
grid is not split, so there is no data-path exchange): its whole-job rate is
the units of all ranks over the slowest rank's time. Checked with two gloo
ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    seconds = 1.0 + rank            # rank 1 is the slowest
    rate = bench.whole_job_rate(dist, torch, 600.0, seconds, ws)
    slow = bench.allmax(dist, torch, seconds)
    bench.barrier(dist, torch)
    out[rank] = (rate, slow)
    dist.destroy_process_group()


def test_whole_job_rate_two_ranks():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        rate, slow = res[r]
        assert slow == 2.0
        assert rate == pytest.approx(600.0 * ws / 2.0)


def test_single_process_rate():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.whole_job_rate(None, torch, 300.0, 1.5, 1) == pytest.approx(200.0)
