"""The bench's multi-rank logic on CPU: two gloo ranks (one process each, as
torchrun launches them) meet at the timing barriers, take the largest of the
ranks' timed seconds and report the whole-job rate; the reference arm runs on
rank 0 only.  No GPU is used."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_on()
        bench.dist_barrier()
        seconds = 1.0 + 0.5 * rank                      # rank 1 is the slower one
        tmax = bench.max_over_ranks(seconds, "cpu")
        rate = bench.whole_job_rate(world, 1000, 4, tmax)
        bench.dist_barrier()
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r\n" % (tmax, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        tmax, rate = (float(x) for x in open(tmp_path / ("rank%d.txt" % r)).read().split())
        assert tmax == 1.5                               # the max over ranks, seen by every rank
        assert rate == pytest.approx(world * 1000 * 4 / 1.5)


def test_single_process_helpers_are_identities():
    sys.path.insert(0, ROOT)
    import bench
    assert not bench.dist_on()
    bench.dist_barrier()
    assert bench.max_over_ranks(2.5, "cpu") == 2.5
    assert bench.whole_job_rate(1, 10, 3, 2.0) == 15.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        config = "tgv16_p4"
        warmup, steps, newton, gpus = 1, 1, 2, 2
    bench.run_reference(Args())                          # returns at once on rank 1
    assert capsys.readouterr().out == ""
