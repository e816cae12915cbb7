"""bench.py's multi-rank path on the CPU (gloo, world size 2, 127.0.0.1):
the whole-job step time is the maximum over ranks, every rank transforms its
own batch (disjoint seeds), and the reference arm under torchrun runs and
prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, timeout=240):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_port())] + args
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_max_over_ranks_without_group():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5


def test_batch_seeds_disjoint_across_ranks():
    import bench
    seen = set()
    for rank in range(8):
        s = bench.batch_seeds(rank, 64)
        assert len(s) == 64 and not seen & set(s)
        seen |= set(s)


def test_gloo_two_ranks_take_the_slowest_step():
    lines = _torchrun([os.path.join("tests", "_ranks_child.py")])
    assert len(lines) == 1  # rank 0 only
    out = json.loads(lines[0])
    assert out["world"] == 2
    assert [r["max"] for r in out["ranks"]] == [15.0, 15.0]
    s0, s1 = (set(map(tuple, r["seeds"])) for r in out["ranks"])
    assert len(s0) == len(s1) == 4 and not s0 & s1


def test_reference_arm_prints_on_rank_zero_only():
    lines = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
                       "--nside", "8", "--lmax", "16", "--maps", "2", "--cpu-rings", "8"])
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
