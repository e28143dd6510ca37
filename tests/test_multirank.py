"""The bench's multi-rank host logic on CPU: two gloo ranks (replicas, weak
scaling) agree on the max and sum reductions the job-level numbers use, draw
different roots, and under torchrun the reference arm prints exactly one line
from rank 0 while rank 1 exits cleanly without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["SS_ROOT"])
import bench, graphgen as gg
world, rank, local, pg = bench.dist_setup()
assert world == 2 and pg is not None
bench.barrier(pg)
mx = bench.max_over_ranks(pg, float(rank + 1))
sm = bench.sum_over_ranks(pg, float(rank + 1))
g = gg.kronecker(8, seed=1)
roots = gg.roots(g, 4, seed=2 + 1000 * rank)
print(json.dumps({"rank": rank, "max": mx, "sum": sm, "roots": [int(r) for r in roots]}), flush=True)
pg.destroy_process_group()
"""


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_and_draw_distinct_roots():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), SS_BENCH_GLOO="1", SS_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["max"] == 2.0 and o["sum"] == 3.0
    assert outs[0]["roots"] != outs[1]["roots"]  # each replica runs its own roots


def test_reference_arm_under_torchrun_prints_one_line():
    port = free_port()
    env = dict(os.environ, SS_BENCH_GLOO="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--scale", "10",
           "--roots", "2", "--ref-seconds", "0.2"]
    r = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
