"""The benchmark's multi-rank bookkeeping (torchrun, one replica per rank) on
CPU with the gloo backend and two ranks: the max-over-ranks timing reduction
and the barrier that bracket the timed region."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
ws, rank, local = bench.dist_env()
assert ws == 2 and rank in (0, 1)
bench.barrier(ws)
t = bench.reduce_max(1.5 + rank, ws)       # rank 1 is the slow one
print(json.dumps({{"rank": rank, "max": t}}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_reduce_max_and_barrier_two_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed unavailable")
    script = tmp_path / "child.py"
    script.write_text(CHILD.format(root=ROOT))
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=240) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
    import json
    vals = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    assert sorted(v["rank"] for v in vals) == [0, 1]
    assert all(v["max"] == 2.5 for v in vals)


def test_reference_arm_exits_cleanly_on_nonzero_rank():
    """Under torchrun only rank 0 runs the reference arm; other ranks exit 0."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


@pytest.mark.slow
def test_reference_arm_prints_the_contract_line():
    """Rank 0 of the reference arm times the FP64 oracle on the host cores (a
    bounded subsample of the N = 2^20 workload) and prints one JSON line with
    the keys the benchmark contract names."""
    import json
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["config"]["workload"].startswith("plummer_n1048576")
