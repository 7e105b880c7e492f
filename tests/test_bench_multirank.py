"""The benchmark's multi-rank logic on CPU, two gloo ranks.

Each rank must draw an independent scene of the same shape and size (weak
scaling with no data exchanged), every rank must agree on the slowest rank's
time, and the reference arm must do its work on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w, r, _ = bench.dist_env()
    sc, dt, batched = bench.make_workload("four_bodies", r)
    s = sc[0]
    slowest = bench.max_over_ranks(1.5 * (r + 1), w)
    dist.barrier()
    rec = {"rank": r, "ws": w, "n": int(s.n), "n_bodies": int(s.n_bodies), "h": s.h, "seed": s.info["seed"],
           "x0": s.x[:4].tolist(), "slowest": slowest, "batched": batched, "dtype": np.dtype(dt).name}
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump(rec, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_draw_independent_equal_size_scenes(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["ws"] == r1["ws"] == 2
    # the same workload shape on both ranks ...
    for k in ("n", "n_bodies", "h", "batched", "dtype"):
        assert r0[k] == r1[k], k
    # ... but an independent draw
    assert r0["seed"] != r1["seed"]
    assert r0["x0"] != r1["x0"]
    # both see the slowest rank's time
    assert r0["slowest"] == r1["slowest"] == 3.0


def test_max_over_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(2.25, 1) == 2.25


def test_reference_arm_runs_on_rank0_only():
    """Under torchrun a rank other than 0 exits 0 at once without output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_json_line():
    """The reference arm (the FP64 oracle on the host cores) prints one JSON
    line with the contract's keys: the metric and unit of the GPU arm, a
    cpu_baseline describing the run, and an e2e block that moves no bytes."""
    import json

    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "two_cubes", "--steps", "2", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "contact particle-iters/s" and d["value"] > 0
    assert d["warmup"] >= 3 and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0 == d["e2e"]["d2h_bytes_per_step"]
    assert "workload" in d["config"]
