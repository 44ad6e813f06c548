"""The N > 1 path of bench.py on the CPU (gloo, two ranks).

With N GPUs the benchmark runs N independent replicas of the workload (the
method does not shard one graph; no collective on the data path).  The job's
time is the slowest rank's, and the rate counts every rank's units.  Also:
the reference arm runs on rank 0 only; other ranks exit at once.
"""
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
total_ms = [120.0, 200.0][rank]          # this rank's timed total
units = 10                               # solves per rank
out = {{"rank": rank,
        "max": bench.max_over_ranks(total_ms, world, "cpu"),
        "rate": bench.whole_job_rate(units, total_ms, world, "cpu")}}
dist.barrier()
dist.destroy_process_group()
print(json.dumps(out), flush=True)
"""


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_replicas_take_the_slowest_rank_and_count_every_rank():
    import json
    port = free_port()
    code = WORKER.format(root=ROOT)
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE="2", LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=120)
        finally:
            if p.poll() is None:
                p.kill()
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for r in outs:
        assert r["max"] == 200.0                       # the slowest replica
        assert r["rate"] == pytest.approx(2 * 10 / 0.200)  # both ranks' solves per second


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""                      # no line, no work on other ranks


def test_kernel_fingerprint_ignores_comments_only(tmp_path, monkeypatch):
    """The profile's code hash survives comment and whitespace edits, not code edits."""
    sys.path.insert(0, ROOT)
    import bench
    a = tmp_path / "a.cu"
    a.write_text("// head\nint f(int x) { /* note */ return x + 1; }\n")
    monkeypatch.setattr(bench, "PROFILED_SOURCES", [str(a)])
    h0 = bench.kernel_fingerprint()
    a.write_text("// another comment\nint f(int x)  {\n  return x + 1;  // trailing\n}\n")
    assert bench.kernel_fingerprint() == h0
    a.write_text("int f(int x) { return x + 2; }\n")
    assert bench.kernel_fingerprint() != h0
