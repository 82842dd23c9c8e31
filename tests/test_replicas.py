"""The multi-rank host path of bench.py on CPU (gloo, world size 2, ranks
as separate processes): the barrier, the maximum over ranks, disjoint input
shards per rank, and the reference arm printed by rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import argparse, json, sys
import torch
import bench, synth
args = argparse.Namespace(impl="reference", workload="plain", steps=1, warmup=3, gpus=2, ref_step_s=0.05)
world, rank, local = bench.dist_setup(args)
bench.barrier(world)
m = bench.max_over_ranks(1.5 * (rank + 1), world, "cpu")
w = synth.PLAIN
B = w.binary()
S = w.samples(B, device="cpu", n=256, start=bench.shard_start(rank, w.n_samples))
json.dump({"rank": rank, "world": world, "max": m, "pc": S.pc.tolist()}, open(sys.argv[1] + f"/r{rank}.json", "w"))
bench.run_reference(args, world, rank)
bench.barrier(world)
torch.distributed.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks(tmp_path, oracle_lib):
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE="2",
                   LOCAL_RANK=str(r))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, str(tmp_path)], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            outs.append(p.communicate(timeout=300))
        finally:
            if p.poll() is None:
                p.kill()
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    assert [x["world"] for x in res] == [2, 2]
    assert [x["max"] for x in res] == [3.0, 3.0]
    assert res[0]["pc"] != res[1]["pc"]                 # each rank its own slice of the stream
    lines = [l for l in outs[0][0].splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["config"]["workload"] == "plain-1M"
    assert not [l for l in outs[1][0].splitlines() if l.startswith("{")]   # rank 1 prints nothing
