"""The multi-process path of bench.py on the host: two ranks under torch.distributed
with the gloo backend (no GPU).  Each rank runs its own lattice in the benchmark
(independent lattices, no data-path collective); what crosses ranks is the
barrier, the max-over-ranks time and the rank-0-only output, tested here."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, sys, types
sys.path.insert(0, sys.argv[1])
import torch
import torch.distributed as dist
import bench

world, rank, local = bench.dist_env()
dist.init_process_group("gloo")
out = {"rank": rank, "world": world, "local": local}
# The slowest rank's time wins; every rank gets the same number.
out["max"] = bench.max_over_ranks(10.0 + rank, torch, world)
bench.barrier(world)
out["mlups"] = bench.aggregate_mlups(world, 4096 * 4096, 100, out["max"])
dist.destroy_process_group()
# The reference arm under the same launcher: rank 0 alone runs it and prints.
args = types.SimpleNamespace(steps=2, warmup=3, gpus=world, layout="rows")
print("RESULT " + json.dumps(out), flush=True)
bench.run_reference(args)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks():
    pytest.importorskip("torch")
    import oracle

    oracle.build()
    port = str(_free_port())
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=port, WORLD_SIZE="2", RANK=str(rank),
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        so, se = p.communicate(timeout=300)
        assert p.returncode == 0, se
        outs.append(so)
    results, lines = [], []
    for so in outs:
        res = [json.loads(l[7:]) for l in so.splitlines() if l.startswith("RESULT ")]
        assert len(res) == 1
        results.append(res[0])
        lines.append([json.loads(l) for l in so.splitlines() if l.startswith("{")])
    for r in results:
        assert r["world"] == 2 and r["max"] == 11.0
        assert r["mlups"] == pytest.approx(2 * 4096 * 4096 * 100 / 11e-3 / 1e6)
    by_rank = {r["rank"]: l for r, l in zip(results, lines)}
    assert len(by_rank[0]) == 1 and by_rank[0][0]["impl"] == "reference" and by_rank[0][0]["value"] > 0
    assert by_rank[1] == []
