"""The multi-process launch path of bench.py on CPU: two gloo ranks started
by torch.distributed.run; only rank 0 prints the JSON line, every rank exits 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_under_two_gloo_ranks():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", MASTER_ADDR="127.0.0.1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29533", "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3", "--cpu-sample-log2", "16"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_rank_helpers_with_gloo(tmp_path):
    code = r"""
import os, sys
sys.path.insert(0, %r)
import torch.distributed as dist
import bench
world, rank, local = bench.dist_setup()
bench.barrier(world)
m = bench.max_over_ranks(float(rank + 1) * 1.5, world)
assert m == 3.0, m
dist.destroy_process_group()
open(os.path.join(%r, "rank%%d.ok" %% rank), "w").write("ok")
""" % (ROOT, str(tmp_path))
    script = tmp_path / "ranks.py"
    script.write_text(code)
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29534", str(script)]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert sorted(p.name for p in tmp_path.glob("rank*.ok")) == ["rank0.ok", "rank1.ok"]
