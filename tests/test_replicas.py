"""The N > 1 path of bench.py (replicas only): world-size-2 gloo ranks on the CPU.

The path shards over independent images with no exchange step (bench.py --gpus N runs
N replicas on disjoint batches); the only cross-rank operation is the MAX of the elapsed
time, and the whole-job throughput counts every rank's units over the slowest rank's time.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 + 5.0 * rank            # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local, world, "cpu")
    value = bench.job_throughput(4, world, ms)
    seeds = list(range(bench.replica_seed0(rank, 4), bench.replica_seed0(rank, 4) + 4))
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"ms": ms, "value": value, "seeds": gathered}, fh)


def test_max_over_ranks_and_throughput_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r in res:
        assert r["ms"] == 15.0                                  # the slowest rank's time on every rank
        assert r["value"] == pytest.approx(4 * 2 / 0.015)       # all ranks' units over that time
    s0, s1 = res[0]["seeds"]
    assert not set(s0) & set(s1) and len(s0) == len(s1) == 4   # disjoint images per replica


def test_single_rank_is_a_no_op():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_throughput(32, 1, 1000.0) == pytest.approx(32.0)


def test_reference_arm_under_torchrun_prints_one_line():
    """Under torchrun with two ranks the reference arm runs on rank 0 alone, which prints the
    single JSON line; rank 1 exits 0 without work."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--workload", "service", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
