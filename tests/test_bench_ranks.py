"""The bench's multi-process host logic on the CPU (gloo, world size 2):
the whole-job rate takes the slowest rank's time and counts every rank's
units; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    per_rank_ms = [400.0, 1000.0][rank]          # rank 1 is the slow one
    rate, t = bench.job_rate(per_rank_ms, 200, world, dist, device="cpu")
    out.put((rank, rate, t))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_is_all_units_over_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, t in res:
        assert t == 1000.0                       # max over ranks
        assert abs(rate - 2 * 200 / 1.0) < 1e-9  # 400 steps in 1 s


def test_single_rank_rate_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    rate, t = bench.job_rate(250.0, 50, 1)
    assert t == 250.0 and abs(rate - 200.0) < 1e-9


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.argparse.Namespace(steps=3, warmup=3, gpus=2)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
