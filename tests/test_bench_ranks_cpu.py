"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): replicas each time
their own steps; the job time is the maximum over ranks and the job rate counts the
units of every rank; the oracle arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r timed 10 * (r + 1) ms over 5 steps of 100 units each
    t_max, value = bench.job_rate(10.0 * (rank + 1), 5, 100, world, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{t_max!r} {value!r}\n")


def test_job_rate_max_over_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        t_max, value = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert t_max == 20.0  # the slower rank decides the job time on every rank
        assert value == pytest.approx(world * 5 * 100 / 0.020)


def test_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench

    t_max, value = bench.job_rate(4.0, 2, 1000, 1)
    assert t_max == 4.0 and value == pytest.approx(2 * 1000 / 0.004)


def test_reference_arm_nonzero_rank_exits_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")

    def boom(*a, **k):  # rank 1 must not run the oracle
        raise AssertionError("oracle run on rank 1")

    monkeypatch.setattr(bench, "oracle_sample", boom)

    class Args:
        steps, warmup, gpus = 1, 0, 2

    assert bench.run_reference(Args()) == 0
