"""Host-side multi-process logic of bench.py (replicas, one per GPU) with two
gloo ranks on the CPU: rank discovery from the environment, the max-over-ranks
reduction of the timed span and the barrier.  No GPU involved."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import bench
    w, r, l, pg = bench.dist_setup(None)
    assert pg is not None and w == world and r == rank
    m = bench.reduce_max(pg, float(10 * (rank + 1)), torch.device("cpu"))
    bench.barrier(pg, torch.device("cpu"))
    with open(os.path.join(out, f"r{rank}.json"), "w") as f:
        json.dump({"rank": r, "world": w, "max": m}, f)
    pg.destroy_process_group()


def test_two_gloo_ranks_reduce_and_barrier(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"r{k}.json")) for k in range(2)]
    assert [r["rank"] for r in res] == [0, 1]
    assert all(r["world"] == 2 and r["max"] == 20.0 for r in res)


def test_reference_arm_prints_one_json_line():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "atom-steps/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["config"]["atoms"] == 1048576 and d["steps"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0
