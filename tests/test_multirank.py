"""The multi-process host logic of bench.py on CPU, two ranks over gloo.

Each GPU runs an independent replica of the solve (the single-system solve
is not partitioned), so the only cross-rank steps are the barriers around
the timed region and the maximum of the ranks' times; rank 0 alone prints,
and the oracle arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, sys
sys.path.insert(0, {root!r})
import bench
ranks, dist = bench.init_ranks("gloo")
bench.barrier(dist)
t = bench.job_seconds(1.5 + ranks.rank, dist, "cpu")
bench.barrier(dist)
print(json.dumps({{"rank": ranks.rank, "world": ranks.world, "local": ranks.local, "t": t}}))
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_env(rank, world, port):
    env = dict(os.environ)
    env.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
               WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return env


def test_job_time_is_the_max_over_two_gloo_ranks():
    port = free_port()
    code = WORKER.format(root=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], env=rank_env(r, 2, port),
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    assert [(d["rank"], d["world"], d["local"]) for d in outs] == [(0, 2, 0), (1, 2, 1)]
    assert [d["t"] for d in outs] == [2.5, 2.5]


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(env={})
    assert (r.world, r.rank, r.local) == (1, 0, 0)
    assert bench.job_seconds(3.25, None) == 3.25


def test_only_rank_zero_prints(capsys):
    sys.path.insert(0, ROOT)
    import bench
    bench.emit({"value": 1.0}, bench.Ranks(env={"RANK": "1", "WORLD_SIZE": "2"}))
    assert capsys.readouterr().out == ""
    bench.emit({"value": 1.0}, bench.Ranks(env={"RANK": "0", "WORLD_SIZE": "2"}))
    assert json.loads(capsys.readouterr().out) == {"value": 1.0}


def test_reference_arm_runs_on_rank_zero_only():
    """Rank 1 of a two-rank launch of the oracle arm exits 0 without work."""
    env = rank_env(1, 2, free_port())
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""
