"""The multi-rank path of bench.py on CPU: two gloo ranks (world_size 2).

Every rank solves its own replica of the batched workload with no collective
on the data path; the only exchange is the end-of-run reduction (slowest
rank's time, observations of all replicas), which these tests run through the
same helper bench.py uses, over gloo instead of NCCL."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank, world, local = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=world)
try:
    ms = [12.5, 17.25][rank]
    units = [1000, 2345][rank]
    t, n = bench.over_ranks(ms, units, world, dist, "cpu")
    specs = bench.sg.batch_c3_specs(replica=rank, n_clusters=8)
    print(json.dumps({{"rank": rank, "world": world, "local": local, "t": t, "n": n, "specs": specs}}))
finally:
    dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(world):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r), WORLD_SIZE=str(world),
                   LOCAL_RANK=str(r), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    out = []
    for p in procs:
        so, se = p.communicate(timeout=180)
        assert p.returncode == 0, se[-2000:]
        out.append(json.loads(so.strip().splitlines()[-1]))
    return out


def test_two_gloo_ranks_reduce_time_and_units():
    res = _run_ranks(2)
    for r, o in enumerate(res):
        assert (o["rank"], o["world"], o["local"]) == (r, 2, r)
        assert o["t"] == 17.25          # the slowest rank's time
        assert o["n"] == 1000 + 2345    # the units of both replicas
    # each rank generates its own replica (distinct sizes and sub-seeds)
    assert res[0]["specs"] != res[1]["specs"]
    assert len(res[0]["specs"]) == len(res[1]["specs"]) == 8


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.over_ranks(3.5, 42, 1) == (3.5, 42)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm's other ranks exit 0 without work."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_reference_arm_prints_its_line_on_rank_zero():
    """The reference arm (the FP64 oracle timed on the host cores) on rank 0
    of a one-rank job prints one JSON line with the value, the cores it used
    and an end-to-end figure without device copies."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--clusters", "2",
                        "--steps", "1", "--warmup", "0", "--iters", "2"], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.strip().splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    o = json.loads(lines[0])
    assert o["impl"] == "reference" and o["value"] > 0 and o["unit"] == "obs/s"
    assert o["cpu_baseline"]["kind"] == "oracle" and o["cpu_baseline"]["cores"] >= 1
    assert o["cpu_baseline"]["value"] == o["value"]
    assert o["e2e"]["value"] == o["value"]
    assert o["e2e"]["h2d_bytes_per_step"] == 0 and o["e2e"]["d2h_bytes_per_step"] == 0
    assert o["config"]["global_batch"] == 2 and o["steps"] == 1 and o["warmup"] == 0
