"""The multi-process path of bench.py on CPU: world size 2 with the gloo backend.

bench.py runs one replica per GPU (targets and (alpha, k) pairs are
independent; there is no data-path collective); the only cross-rank step is
the max over ranks of the step times, and the reported value is all ranks'
units over the slowest rank's time.  The reference arm runs on rank 0 only.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = """
import json, sys
import torch.distributed as dist
sys.path.insert(0, {root!r})
import bench
dist.init_process_group("gloo")
r = dist.get_rank()
print(json.dumps(bench.max_over_ranks([1.0 + r, 10.0 - r, 0.5 * r])))
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert outs[0] == outs[1] == [2.0, 10.0, 0.5]


def test_single_rank_is_identity_and_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.whole_job_rate(10**6, 2, 0.5) == 4e6


def test_replica_clouds_differ_by_rank():
    from paper_1801_05977_gb300 import workloads as W
    a, b = W.targets_3d(64, seed=0), W.targets_3d(64, seed=1)
    assert a.shape == b.shape == (64, 3) and not (a == b).all()


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
