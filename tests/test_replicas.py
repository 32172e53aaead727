"""The multi-GPU path of the benchmark without GPUs.  The method's runs
exchange no data, so N GPUs run N independent replicas (one process each);
the host logic is the per-rank replica configuration and the whole-job
aggregate: the slowest rank's time and the sum of all ranks' particle-steps.
Here two ranks run that aggregate over gloo on CPU, and the reference arm is
checked to run on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    # rank r: 10 + r ms for (r + 1) * 1000 particle-steps
    t, ps = bench.job_totals(10.0 + rank, 1000.0 * (rank + 1), world)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"t": t, "ps": ps}, f)


def test_job_totals_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        got = json.load(open(tmp_path / ("rank%d.json" % r)))
        assert got == {"t": 11.0, "ps": 3000.0}  # every rank sees the job's totals


def test_single_rank_totals_are_its_own():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_totals(12.5, 4000.0, 1) == (12.5, 4000.0)


def test_replicas_are_independent_runs():
    sys.path.insert(0, ROOT)
    import bench
    cfg = dict(workloads.CFG_WIDE_EXPLICIT)
    r0, r1 = bench.replica_config(cfg, 0), bench.replica_config(cfg, 1)
    assert (r0["seed"], r0["run"]) != (r1["seed"], r1["run"])
    assert {k: v for k, v in r0.items() if k not in ("seed", "run")} == \
           {k: v for k, v in r1.items() if k not in ("seed", "run")}


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env = dict(os.environ, RANK="0", WORLD_SIZE="2", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
