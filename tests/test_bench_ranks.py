"""The multi-rank logic of bench.py on the CPU: two gloo ranks run the
barrier, the max-over-ranks reduction and the whole-job rate of independent
replicas (the path has no data exchange between GPUs: replicas only), and
the reference arm leaves every rank but 0 without work and on rank 0 prints
one JSON line for the native arm's metric and workload."""
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
dist.init_process_group("gloo", init_method="env://")
import bench
world, rank, _ = bench.dist_env()
bench.barrier(world)
m = bench.max_over_ranks(world, 1.0 + rank)
rate, t = bench.job_rate(world, 100, 2.0 if rank == 0 else 4.0)
print(json.dumps({{"rank": rank, "world": world, "max": m, "rate": rate, "t": t}}), flush=True)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_ranks(code, world=2, extra_env=None, timeout=120):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="", **(extra_env or {}))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=timeout)
        except subprocess.TimeoutExpired:
            p.kill()
            out, err = p.communicate()
        outs.append((p.returncode, out, err))
    return outs


def test_two_gloo_ranks_reduce_and_aggregate():
    import json
    outs = _run_ranks(CHILD.format(root=ROOT))
    for rc, out, err in outs:
        assert rc == 0, err
    lines = [json.loads(o.strip().splitlines()[-1]) for _, o, _ in outs]
    for d in lines:
        assert d["world"] == 2
        assert d["max"] == 2.0                 # max over ranks of 1 + rank
        assert d["t"] == 4.0                   # the slowest rank's time
        assert d["rate"] == pytest.approx(2 * 100 / 4.0)


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm's rank 1 exits 0 without work (rank 0
    is not started here: it would time the oracle for a minute)."""
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_candidate_pairs_counts_the_full_stencil():
    """The issued-work count of the bench: every ordered pair (i, j) whose
    cells are within k cells of each other on the periodic grid, self pairs
    included, checked by brute force over particles on small grids."""
    import itertools
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(3)
    for nc, k in ((5, 1), (6, 2), (3, 1)):
        g = rng.integers(0, 4, size=(nc, nc, nc))
        cells = [c for c in itertools.product(range(nc), repeat=3) for _ in range(g[c])]
        brute = 0
        for a in cells:
            for b in cells:
                d = [min((a[i] - b[i]) % nc, (b[i] - a[i]) % nc) for i in range(3)]
                brute += max(d) <= k
        assert bench.candidate_pairs(torch.from_numpy(g).double(), k) == brute


@pytest.mark.slow
def test_reference_arm_line():
    """The reference arm (the oracle on the host cores) prints one JSON line
    with the native arm's metric, unit and workload, the requested warm-up
    steps (at least 3), a cpu_baseline describing the run and an e2e entry
    with no host-device bytes."""
    import json
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    for key in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        env.pop(key, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "steps/s"
    assert d["config"]["workload"] == bench.WORKLOAD and d["config"]["n"] == 4_000_000
    assert d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
