"""bench.py's multi-rank path on CPU: two gloo ranks, one process each with
the environment torchrun gives them.  Checks the max-over-ranks timing rule,
the barrier, the whole-job rate (units of all ranks / slowest time), and that
only rank 0 of the reference arm does work."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
world, rank = bench.dist_setup()
t = bench.max_over_ranks(1.0 + rank, world)   # rank r "took" 1 + r ms
bench.barrier(world)
print(json.dumps({{"rank": rank, "world": world, "max_ms": t,
                   "value": bench.whole_job_rate(1000, world, t)}}))
import torch.distributed as dist
dist.destroy_process_group()
"""


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ)
    env.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
    return env


def test_two_gloo_ranks(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(RANK_SCRIPT.format(root=ROOT))
    port = _port()
    procs = [subprocess.Popen([sys.executable, str(script)], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["world"] == 2
        assert o["max_ms"] == 2.0                 # the slowest rank's time
        assert o["value"] == 2 * 1000 / 2e-3      # all ranks' units / that time
    assert sorted(o["rank"] for o in outs) == [0, 1]


def test_reference_arm_runs_on_rank_zero_only():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], env=_env(1, 2, _port()), capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
