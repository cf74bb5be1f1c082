"""The multi-rank path of bench.py on CPU: two gloo ranks (world size 2, 127.0.0.1) run the
replica bookkeeping the GPU ranks run (per-rank seeds, the slowest rank's time, whole-job
throughput), and the reference arm under a launcher leaves every rank but 0 without work."""
import os
import socket
import subprocess
import sys

import pytest

from conftest import ROOT

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(4, rank))
        ms = 10.0 + 5.0 * rank                      # rank 1 is the slower one
        ms_max = bench.max_over_ranks(ms, dist)
        out[rank] = (seeds, ms_max, bench.job_rate(3624, world, ms_max))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        seeds, ms_max, rate = res[rank]
        assert len(set(seeds)) == world             # independent fields per rank
        assert ms_max == 15.0                       # every rank sees the slowest rank's time
        assert rate == pytest.approx(2 * 3624 / 0.015)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, None) == 7.5
    assert bench.job_rate(100, 1, 10.0) == pytest.approx(1e4)


def test_reference_arm_on_other_ranks_does_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
