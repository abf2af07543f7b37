"""The multi-process form on CPU (gloo, world size 2): the workload runs as
independent replicas per rank (no collective on the data path), the step time is
the maximum over ranks, and under torchrun only rank 0 prints a line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_max = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        seeds = bench.replica_seeds(rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        with open(out + f".{rank}", "w") as f:
            json.dump({"t_max": t_max, "seeds": gathered}, f)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_replica_seeds_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world, port, out = 2, _free_port(), str(tmp_path / "r")
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for rank in range(world):
        r = json.load(open(out + f".{rank}"))
        assert r["t_max"] == 2.5  # the slower rank's time, on every rank
        s0, s1 = r["seeds"]
        assert len(s0) == len(bench.SEEDS) and not set(s0) & set(s1)  # independent chains per rank
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25


def test_reference_arm_under_torchrun_prints_once():
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1  # rank 0 only
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
