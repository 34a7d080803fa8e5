"""The N > 1 bench path (replicas only: one independent solve per rank, no
collective on the data path) aggregated over two gloo ranks on the CPU: the job
time is the slowest rank's and the value counts the dofs of every rank."""
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


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms = [120.0, 80.0][rank]                     # rank 0 is the slow one
    job_ms, value = bench.aggregate_replicas(ms, 1_000_000, 10, dist, "cpu")
    q.put((rank, job_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, job_ms, value in out:
        assert job_ms == 120.0
        # 2 ranks x 10 solves x 1e6 dofs in 0.12 s
        assert value == pytest.approx(2 * 10 * 1e6 / 0.12 / 1e6)


def test_single_process_aggregation():
    sys.path.insert(0, ROOT)
    import bench
    job_ms, value = bench.aggregate_replicas(50.0, 2_000_000, 5)
    assert job_ms == 50.0 and value == pytest.approx(5 * 2.0 / 0.05)
