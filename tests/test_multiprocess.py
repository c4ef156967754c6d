"""The N > 1 path of bench.py on the CPU: two gloo ranks, replicas only.

Each rank solves its own pair; the only communication is the timing reduction:
the job rate is the units of all ranks over the slowest rank's time."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        ranks = bench.Ranks(world, "cpu")
        ranks.barrier()
        # rank r processed 10 + r units in 100 * (r + 1) ms
        rate = bench.whole_job_rate(ranks, 10.0 + rank, 100.0 * (rank + 1))
        out[rank] = (ranks.max(float(rank)), ranks.sum(1.0), rate)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_weak_scaling_reduction():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        mx, total, rate = res[r]
        assert mx == 1.0 and total == 2.0
        # (10 + 11) units over the slowest rank's 0.2 s
        assert rate == pytest.approx(21.0 / 0.2)


def test_single_rank_needs_no_process_group():
    bench = _bench()
    ranks = bench.Ranks(1, "cpu")
    ranks.barrier()
    assert ranks.max(3.0) == 3.0 and ranks.sum(3.0) == 3.0
    assert bench.whole_job_rate(ranks, 5.0, 500.0) == pytest.approx(10.0)
