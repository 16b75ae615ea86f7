"""The N > 1 path of bench.py on CPU: two gloo ranks, each a replica with its own
measured time; the line must use the slowest rank's time and count every rank's node
updates, and the reference arm must run on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    d.init("gloo")
    my_ms = 100.0 + 25.0 * rank          # rank 1 is the slow replica
    d.barrier()
    worst = d.max(my_ms)
    value = bench.whole_job_mlups(d.world, 1000, 50, worst)
    d.close()
    q.put((rank, worst, value))


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, worst, value in out:
        assert worst == 125.0
        assert value == pytest.approx(2 * 1000 * 50 / 0.125 / 1e6)


def test_reference_arm_prints_on_rank_zero_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload, steps, warmup = "couette", 3, 3

    bench.reference(A())
    assert capsys.readouterr().out == ""
