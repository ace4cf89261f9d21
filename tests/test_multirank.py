"""The benchmark's multi-rank path (one process per GPU, max over ranks,
rank 0 reports) on CPU with two gloo ranks; the reference arm's non-zero
ranks exit without work."""
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


def _rank_main(rank, ws, port, q):
    os.environ.update({"WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    g = bench.RankGroup("gloo")
    g.barrier()
    got = g.max(1.5 + rank)              # per-rank time; the job takes the slowest
    q.put((rank, g.ws, got))
    g.close()


def test_two_gloo_ranks_take_the_max():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(ws))
    assert res == [(0, 2, 2.5), (1, 2, 2.5)]


def test_reference_arm_nonzero_rank_exits_without_work(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    sys.path.insert(0, ROOT)
    import bench

    class A:
        level, k, steps, warmup, ref_rows = 7, 50.0, 3, 1, 384
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
