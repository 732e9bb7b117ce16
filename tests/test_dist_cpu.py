"""The N > 1 path of bench.py on CPU: two processes under
torch.distributed.run with the gloo backend (replicas only: no data-path
collective; the ranks exchange one timing value for the max over ranks)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def torchrun(args, timeout=300):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port())] + args
    env = dict(os.environ, OMP_NUM_THREADS="2")
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def json_lines(out: str):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_replica_aggregation_gloo_world_size_2(tmp_path):
    r = torchrun([os.path.join("tests", "gloo_rank.py"), str(tmp_path)])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads((tmp_path / f"rank{k}.json").read_text()) for k in range(2)]
    assert [d["rank"] for d in lines] == [0, 1]
    for d in lines:
        assert d["ws"] == 2
        assert d["t_max"] == 15.0  # the slowest replica's time on every rank
        assert d["value"] == 1.0e9 * 2 / 0.015  # all ranks' work over the slowest time
    assert lines[0]["seed"] != lines[1]["seed"]  # each replica evolves its own lattice


def test_reference_arm_prints_once_under_torchrun():
    r = torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1  # rank 0 alone runs and prints; rank 1 exits 0 without work
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
