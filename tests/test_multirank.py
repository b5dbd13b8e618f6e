"""The replica path of bench.py on two CPU ranks over gloo: each rank solves
its own system, the job time is the slowest rank's, the value sums the ranks'
rows.  No GPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [2.0, 3.5][rank]
    bench.barrier(world)
    job = bench.max_over_ranks(ms, world)
    q.put((rank, job, bench.job_value(1 << 20, world, job)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [3.5, 3.5]
    assert out[0][2] == pytest.approx(2 * (1 << 20) / 3.5e-3)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        n, steps, warmup, gpus = 1 << 10, 1, 1, 2

    bench.reference_arm(A)
    assert capsys.readouterr().out == ""
