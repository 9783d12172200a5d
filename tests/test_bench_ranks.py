"""The multi-rank logic of bench.py on CPU ranks (gloo): replicas, the
slowest rank's time, the whole-job rate, and the reference arm's silence on
ranks other than 0.  No GPU is needed."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(0.5 + rank, dist, "cpu")        # rank r took 0.5 + r seconds
    out[rank] = (t, bench.whole_job_rate(20, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_rate():
    world = 2
    port = free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(rank_main, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    for r in range(world):
        t, rate = got[r]
        assert t == 1.5                              # the slowest of 0.5 and 1.5 s
        assert rate == pytest.approx(2 * 20 / 1.5)   # both replicas' solves per that time


def test_reference_arm_is_silent_on_other_ranks(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        gpus, steps, warmup = 2, 1, 0
    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""
