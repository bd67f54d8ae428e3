"""Multi-process paths on the CPU with the gloo backend (world size 2).

The step does not shard across GPUs: `bench.py --gpus N` runs N independent
replicas, one per rank.  What crosses ranks is the job's timing -- the longest
timed span and the total units processed -- and the reference arm, which rank 0
alone runs and prints.  Both are exercised here without a GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms, units = bench.whole_job(10.0 + 5.0 * rank, 100.0 + rank, dist)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump([ms, units], f)


def test_whole_job_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank, args=(2, free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        with open(os.path.join(tmp_path, f"r{r}.json")) as f:
            ms, units = json.load(f)
        assert ms == 15.0          # the slower rank's span
        assert units == 201.0      # both replicas' units


def test_whole_job_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(12.5, 7, None) == (12.5, 7.0)


def test_reference_arm_under_torchrun():
    """`bench.py --impl reference` launched like the multi-GPU bench: rank 0
    prints one JSON line, the other rank exits 0 without output."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
