"""The multi-process path of bench.py on CPU: two gloo ranks (127.0.0.1)
exercise the whole-job rate (max over ranks of each rank's timed total,
world x steps units), the per-rank right-hand-side seeds of the weak-scaling
replicas, and the reference arm, which only rank 0 runs."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slower one
    ms, rate = bench.job_rate(local_ms, 5, world, dist, "cpu")
    out[rank] = (ms, rate, bench.rank_seed(1000, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_and_seeds_over_two_gloo_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()   # no fork of a multi-threaded process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        ms, rate, seed = out[rank]
        assert ms == 200.0                     # max over ranks
        assert rate == pytest.approx(world * 5 / 0.2)
    assert out[0][2] != out[1][2]              # replicas solve different problems


def test_single_rank_rate():
    ms, rate = bench.job_rate(50.0, 10, 1)
    assert ms == 50.0 and rate == pytest.approx(200.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_prints_one_contract_line():
    """Rank 0 of the reference arm (the oracle on the host cores) prints one
    JSON line with the keys of the benchmark line, no device copies, and the
    same workload as the library's arm."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["n_gpus"] == 1
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["config"]["workload"] == bench.WORKLOAD_NAME
    for key, val in bench.WORKLOAD.items():
        assert d["config"][key] == val, key
