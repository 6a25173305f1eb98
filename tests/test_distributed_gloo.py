"""The multi-rank bench path on CPU with gloo (world size 2): every rank's
elapsed time is gathered, the job time is the slowest rank's, and the value
counts all ranks' units; the reference arm prints one line from rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, result_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank                 # rank 1 is the slower one
    all_ms = bench.dist_max(ms, world)
    value, ms_per_step = bench.aggregate(all_ms, [1000] * world, steps=4)
    bench.barrier(world)
    with open(os.path.join(result_dir, f"r{rank}.json"), "w") as f:
        json.dump({"all": all_ms, "value": value, "ms_per_step": ms_per_step}, f)
    dist.destroy_process_group()


def test_gather_and_aggregate_over_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["all"] == [10.0, 15.0]
        assert r["value"] == pytest.approx(2000 / 15e-3)     # all units over the slowest rank's time
        assert r["ms_per_step"] == pytest.approx(15.0 / 4)


def test_reference_arm_prints_once_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
