"""Multi-rank host logic of bench.py on CPU with the gloo backend (world size 2): every rank runs
its own replica (distinct seeds, no data-path collective), the timed region's maximum over ranks
sets the aggregate rate, and the reference arm prints from rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        local_ms = 10.0 + 5.0 * rank                     # rank 1 is the slow one
        tot = bench.reduce_max(local_ms, "cpu")
        rate = bench.aggregate_steps_per_s(tot, 100, world)
        results[rank] = (tot, rate, bench.replica_seed(2000, rank))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_with_gloo():
    world = 2
    mgr = mp.Manager()
    results = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), results), nprocs=world, join=True)
    (t0, r0, s0), (t1, r1, s1) = results[0], results[1]
    assert t0 == t1 == 15.0                               # max over ranks
    assert r0 == r1 == pytest.approx(2 * 100 / 0.015)      # all ranks' steps over the slowest time
    assert s0 != s1                                       # independent replicas


def test_single_process_needs_no_process_group():
    import bench
    assert not dist.is_initialized()
    assert bench.reduce_max(3.5) == 3.5
    assert bench.aggregate_steps_per_s(1000.0, 50, 1) == pytest.approx(50.0)


def test_reference_arm_runs_on_rank_0_only():
    """Under torchrun the reference arm's non-zero ranks exit 0 without work or output."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=root, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-500:]
    assert r.stdout.strip() == ""
