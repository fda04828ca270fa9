"""The multi-process path of bench.py (CPU, gloo, world size 2): the step
runs as independent replicas, one per rank, and the whole-job rate takes the
slowest rank's time (max over ranks) times the number of ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, rate = bench.job_rate(0.010 + 0.001 * rank, 1000, dist, "cpu")
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{t!r} {rate!r}")
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_over_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        t, rate = (float(x) for x in (tmp_path / f"rank{r}.txt").read_text().split())
        assert t == pytest.approx(0.011)
        assert rate == pytest.approx(world * 1000 / 0.011 / 1e6)


def test_job_rate_single_process():
    import bench
    t, rate = bench.job_rate(0.02, 5000)
    assert t == 0.02 and rate == pytest.approx(5000 / 0.02 / 1e6)
