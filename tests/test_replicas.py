"""Multi-GPU is replicas only (independent pairs, no collective on the data path); the bench
aggregates replicas by the slowest rank's time.  Checked here with 2 gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    q.put((rank, ms, bench.replica_value(world, 20, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_by_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [150.0, 150.0]
    assert out[0][2] == pytest.approx(2 * 20 / 0.150)


def test_replica_value_is_whole_job_throughput():
    import bench
    assert bench.replica_value(1, 20, 1000.0) == pytest.approx(20.0)
    assert bench.replica_value(4, 20, 2000.0) == pytest.approx(40.0)
