"""The reference arm of bench.py (the oracle timed on the host cores) on the
small flat-screen workload: one JSON line with the contract's keys, the same
config text as the GPU arm prints for that workload, and, under two gloo
ranks, one line from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lines(out: str):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "flat",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    sys.path.insert(0, ROOT)
    import bench
    from paper_2310_09204_gb300 import workloads as WL
    # the GPU arm prints the same config for the same workload and N
    assert d["config"] == bench.book_config("flat", WL.flat_config(), 1)
    assert d["cpu_baseline"]["phases_last"]["iters"] > 0
    assert d["cpu_baseline"]["phases_last"]["ndof"] == 225       # the flat screen's dofs


def test_reference_line_serving_stream():
    """The serving workload: each step one full oracle solve of a small request
    of the stream (here a 40-request stream, two steps)."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--serve-requests", "40",
                        "--steps", "2", "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    sys.path.insert(0, ROOT)
    import bench
    assert d["config"] == bench.c5_config(40, 2, 1)
    assert d["value"] > 0 and d["cpu_baseline"]["phases_last"]["iters"] > 0
    assert d["cpu_baseline"]["phases_last"]["ndof"] <= 7000


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_reference_two_ranks_rank0_only():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_port()), "bench.py", "--impl", "reference",
           "--workload", "flat", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
