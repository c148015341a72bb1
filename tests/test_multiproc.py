"""The N > 1 host path, on CPU with world_size-2 gloo process groups.

The chain shards as independent replicas (no data-path collective): each rank
runs the whole workload, the only collective is the max of the per-rank
timings, and rank 0 alone prints the result. Checked here:
  * max_over_ranks returns the per-entry maximum over ranks on every rank;
  * whole_job_rate counts the units of all ranks;
  * bench.py --impl reference under torchrun with 2 ranks prints exactly one
    JSON line (rank 0) and both ranks exit 0.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5 * (rank == 1)], world)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"r{rank}.json"), "w") as fh:
        json.dump(got, fh)


def test_max_over_ranks_gloo_two_ranks(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        with open(tmp_path / f"r{r}.json") as fh:
            assert json.load(fh) == [2.0, 10.0, 0.5]


def test_max_over_ranks_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3, 1.5], 1) == [3.0, 1.5]


def test_whole_job_rate_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    px = 1024 * 1024 * 1500
    one = bench.whole_job_rate(1, px, 10, 2.0)
    assert one == pytest.approx(px * 10 / 2.0 / 1e9)
    assert bench.whole_job_rate(4, px, 10, 2.0) == pytest.approx(4 * one)


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2
    assert rec["value"] > 0 and rec["e2e"]["h2d_bytes_per_step"] == 0
    assert rec["cpu_baseline"]["kind"] == "oracle"
