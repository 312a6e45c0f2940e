"""bench.py's whole-job rate over replicas on a world-size-2 gloo group (CPU):
every rank ends with the slowest rank's time, and the rate counts all ranks'
units over that time (the driver's N > 1 runs use NCCL on GPUs; the
aggregation is the same code)."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        local_ms = 100.0 * (rank + 1)            # rank 1 is the slowest
        dist.barrier()
        total_ms, rate = b.job_rate(torch, dist, torch.device("cpu"), local_ms, world * 10_000 * 5)
        out[rank] = (total_ms, rate)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_job_rate_takes_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    for total_ms, rate in res.values():
        assert total_ms == 200.0
        assert rate == pytest.approx(2 * 10_000 * 5 / 0.2)


def test_job_rate_single_process():
    b = _bench()
    total_ms, rate = b.job_rate(torch, None, None, 50.0, 10_000)
    assert total_ms == 50.0 and rate == pytest.approx(200_000.0)
