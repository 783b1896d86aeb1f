"""The benchmark's multi-GPU contract on CPU: replicas (no data-path
collective), the job time is the slowest rank's, and the value is the sum of
all ranks' node updates over that time.  Two gloo ranks stand in for GPUs."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t_max = bench.max_over_ranks(times[rank], world, "cpu")
    q.put((rank, t_max, bench.replica_mlups(1000, 10, t_max, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [0.5, 0.8]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, v in out:
        assert t_max == 0.8
        assert v == pytest.approx(2 * 1000 * 10 / 0.8 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 3, 3

    assert bench.run_reference(A()) is None
