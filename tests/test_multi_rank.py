"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks run independent replicas (no
data-path collective); the job's time is the maximum over ranks and its throughput counts
every rank's units."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_setup() == (world, rank, rank)
    local_ms = [120.0, 80.0][rank]  # the slower rank decides the job's time
    value, ms = bench.job_rate(local_ms, 1000, world)
    out[rank] = (value, ms)
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    port = 29500 + os.getpid() % 2000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        value, ms = res[rank]
        assert ms == 120.0
        assert value == pytest.approx(2 * 1000 / 0.120)


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench

    value, ms = bench.job_rate(50.0, 500, 1)
    assert ms == 50.0 and value == pytest.approx(500 / 0.05)
