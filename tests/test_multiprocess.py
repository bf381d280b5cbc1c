"""The multi-process (torchrun) path of bench.py on the CPU with the gloo backend, world size 2:
the timing reduction takes the maximum over ranks, the whole-job value counts every rank's
replicas, and the reference arm runs on rank 0 only (the other ranks exit 0 without work)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = 10.0 + 5.0 * rank          # rank 1 is the slow one
    m = bench.max_over_ranks(elapsed, dist)
    v = bench.whole_job_value(m, steps=2, world=world, instances_per_step=2)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, m, v))


def test_max_over_ranks_and_whole_job_value_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 15.0                  # the slowest rank
        assert v == pytest.approx(15.0 / (2 * 2 * 2))


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup, gpus = 1, 0, 2

    def no_work(*a, **k):
        raise AssertionError("rank 1 must not run the oracle")

    monkeypatch.setattr(bench, "OracleKrylovSample", no_work)
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_max_over_ranks_without_a_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
