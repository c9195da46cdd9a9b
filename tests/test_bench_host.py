"""bench.py's multi-rank host logic, run as two gloo ranks on the CPU: the
timed region's slowest-rank time and the whole-job value (each rank
advances its own lattice: replicas, no data-path collective), and the
reference arm's ranks other than 0, which exit without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.getcwd())
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, ws = dist.get_rank(), dist.get_world_size()
ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, device="cpu")
print(json.dumps({"rank": rank, "ms": ms, "value": bench.whole_job_mlups(ws, 1000, 10, ms)}))
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slowest_rank_and_whole_job_value_gloo():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], cwd=ROOT, env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["ms"] == 15.0  # the slower rank's time on every rank
        assert o["value"] == pytest.approx(2 * 1000 * 10 / 15e-3 / 1e6, rel=1e-15)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_mlups(1, 4097 * 4097, 100, 20.0) == pytest.approx(4097 * 4097 * 100 / 0.02 / 1e6)


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
