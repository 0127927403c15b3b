"""The multi-rank arithmetic of bench.py, on CPU with two gloo ranks.

Under torchrun every rank projects its own replica of the workload. The step time of the job is
the slowest rank's (an all-reduce MAX), and the job's throughput counts the tetrahedra of every
rank. The reference arm (the CPU oracle) runs on rank 0 alone.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench

        ms = bench.max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")
        q.put((rank, ms, bench.job_throughput(ws, 1000, ms)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_step():
    import multiprocessing as mp

    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=180) for _ in range(ws))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    assert [r for r, _, _ in res] == [0, 1]
    for _, ms, thr in res:
        assert ms == 15.0  # the slower rank's step
        assert thr == pytest.approx(2 * 1000 / 0.015)  # both ranks' tetrahedra over that step


def test_one_rank_is_its_own_max():
    import bench

    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput(1, 500, 250.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(None)  # returns before reading its arguments
    assert capsys.readouterr().out == ""
