"""The multi-rank host logic of bench.py on CPU: two ranks over gloo.

With N ranks every rank runs its own replica of the workload (weak scaling,
no data-path collective); the job's time is the slowest rank's, taken with a
max-reduction, and the job's rate counts the units of all ranks.  Under
torchrun the reference arm runs on rank 0 only; the other ranks exit 0
without output."""
import os
import socket
import subprocess
import sys
import time

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, delays):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        cpu = torch.device("cpu")
        # a fixed per-rank value: every rank receives the largest
        xs = [1.5, 4.25, 0.5, 3.0][:world]
        got = bench.max_over_ranks(torch, dist, world, xs[rank], cpu)
        assert got == max(xs), (rank, got)
        # a timed region bracketed by barriers: the slower rank sets the time
        dist.barrier()
        t0 = time.perf_counter()
        time.sleep(delays[rank])
        dist.barrier()
        local = time.perf_counter() - t0
        job = bench.max_over_ranks(torch, dist, world, local, cpu)
        assert job >= max(delays) - 1e-3 and job >= local, (rank, job, local)
        # the whole-job rate: all ranks' units over the job's time
        assert abs(bench.job_rate(world, 10.0, job) - world * 10.0 / job) <= 1e-12
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks():
    mp.spawn(_worker, args=(2, _free_port(), [0.0, 0.2]), nprocs=2, join=True)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(torch, None, 1, 2.5, torch.device("cpu")) == 2.5
    assert bench.job_rate(1, 8.0, 2.0) == 4.0
    assert bench.job_rate(4, 8.0, 2.0) == 16.0


def test_reference_arm_other_ranks_exit_silently():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
