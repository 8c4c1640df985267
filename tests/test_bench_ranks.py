"""The multi-process path of the benchmark on CPU (gloo, world size 2): every
rank runs its own replica of the step (no collective on the data path); the
timed region's value is the units of all ranks over the slowest rank's time,
taken with one max-reduction; under the reference arm only rank 0 works."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")   # rank 1 is the slow one
        rate = bench.whole_job_rate(200, world, slowest / 1e3)
        out[rank] = (slowest, rate)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]                                   # every rank reports the same numbers
    slowest, rate = res[0]
    assert slowest == 15.0
    assert rate == pytest.approx(2 * 200 / 0.015)             # both ranks' steps over the slowest time


def test_one_rank_needs_no_collective():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0


def test_reference_arm_other_ranks_exit_without_work(capsys):
    class A:
        n, steps, warmup = 1000, 1, 1
    assert bench.run_reference(A(), 2, 1) is None              # rank 1: returns at once, prints nothing
    assert capsys.readouterr().out == ""


def test_single_line_modes_parse(monkeypatch):
    """`--only batched` defaults to the batched line's workload (2M Gaussians,
    32 views) and takes its size from --batch-n / --batch-views; the default
    run measures the training step (no single-line mode)."""
    monkeypatch.setattr("sys.argv", ["bench.py"])
    a = bench.parse()
    assert a.only is None and a.n == 3_000_000 and a.steps >= 1 and a.warmup >= 3
    monkeypatch.setattr("sys.argv", ["bench.py", "--only", "batched", "--steps", "3", "--warmup", "2"])
    a = bench.parse()
    assert (a.only, a.batch_n, a.batch_views, a.steps, a.warmup) == ("batched", 2_000_000, 32, 3, 2)
    monkeypatch.setattr("sys.argv", ["bench.py", "--only", "batched", "--batch-n", "1000000", "--batch-views", "8"])
    a = bench.parse()
    assert (a.batch_n, a.batch_views) == (1_000_000, 8)
    monkeypatch.setattr("sys.argv", ["bench.py", "--only", "nothing"])
    with pytest.raises(SystemExit):
        bench.parse()
