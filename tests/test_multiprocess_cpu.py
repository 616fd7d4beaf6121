"""The N > 1 launch path on CPU (gloo): rank helpers and the reference arm.

bench.py under torchrun gives each rank its own seeded batch (no collective
on the data path), times with a barrier on both sides and takes the maximum
over ranks; the reference arm runs on rank 0 alone.  Both are exercised
here with two gloo ranks on 127.0.0.1.
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


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from paper_2405_05974_b300 import mechgen, workloads
    r, w, local, pg = bench.dist_setup()
    assert (r, w) == (rank, world) and pg is not None
    bench.barrier(pg)
    mx = bench.max_over_ranks(pg, float(10 + rank))
    # the per-rank batch: the state seed is offset by the rank
    cfg = workloads.STATES["tiny"]
    cfg = type(cfg)(**{**cfg.__dict__, "seed": cfg.seed + 1000 * rank})
    _, T, _ = mechgen.generate_states(workloads.mechanism("tiny"), cfg, 8)
    with open(out % rank, "w") as f:
        json.dump({"max": mx, "T0": float(T[0])}, f)
    pg.destroy_process_group()


def test_rank_helpers_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "rank%d.json")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, start_method="spawn")
    r0 = json.load(open(out % 0))
    r1 = json.load(open(out % 1))
    assert r0["max"] == r1["max"] == 11.0
    assert r0["T0"] != r1["T0"]


def test_reference_arm_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "tiny",
           "--cpu-seconds", "1"]
    p = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
