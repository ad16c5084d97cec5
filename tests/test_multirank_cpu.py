"""The N > 1 host logic of bench.py on CPU: two gloo ranks, each with its own timing,
agree on the slowest rank's time and on the whole-job value (weak scaling); the CPU
reference arm prints only on rank 0."""
import os
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [120.0, 150.0][rank]
    value, t = bench.whole_job_value(local, 500, 10, world, bench.torch_max_reducer("cpu"))
    out[rank] = (value, t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_agree_on_max_time_and_value():
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    value, t = res[0]
    assert t == 150.0
    assert abs(value - 500 * 10 * 2 / 0.150) < 1e-6


def test_reference_arm_prints_only_on_rank_0():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_on_rank_0():
    """The reference arm (the FP64 oracle on the host cores) prints one JSON line with the
    GPU arm's metric, unit and workload, its own cpu_baseline and an e2e with no transfers."""
    import json

    import bench
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0
    assert d["config"]["workload"].startswith("c5: n=1000000 items, m=2000000 users, d=128")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
