"""bench.py's multi-rank timing on CPU with gloo, world size 2: each rank
combs its own copy of the workload, the job time is the slowest rank's, and
the value counts every rank's units (weak scaling)."""
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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 100.0 + 50.0 * rank                  # the ranks took different times
    job = bench.max_over_ranks(local, dist)
    value = bench.weak_scaling_value(1e12, world, 5, job)
    out[rank] = (job, value)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 150.0       # max over ranks
    assert out[0][1] == pytest.approx(1e12 * 2 * 5 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.weak_scaling_value(10.0, 1, 2, 1000.0) == 20.0


def test_reference_arm_line():
    """bench.py --impl reference (the CPU oracle, no GPU) prints one JSON line
    with the contract's keys, its own cpu_baseline and a zero-copy e2e."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--workload", "lcs_dna_512_w16", "--steps", "2", "--warmup", "1",
                        "--ref-seconds", "0.5"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["config"]["workload"] == "lcs_dna_512_w16"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
