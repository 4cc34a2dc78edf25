"""Host-side checks of bench.py (no GPU): the reference arm's JSON line, its
multi-rank behaviour, and the capture digest that decides whether recorded
DRAM traffic is reported."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _json_lines(out):
    return [json.loads(ln) for ln in out.splitlines() if ln.startswith("{")]


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["warmup"] >= 3 and d["steps"] == 1
    assert d["config"]["workload"] == "plain_640x480_var"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_two_ranks_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def test_reference_arm_config_is_the_bench_workload():
    sys.path.insert(0, ROOT)
    import bench
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d, = _json_lines(r.stdout)
    assert d["config"] == bench.bench_config(1)
    assert d["cpu_baseline"]["host_cores"] >= 1 and d["cpu_baseline"]["cpu_model"]


def test_gpus_flag_relaunches_under_torchrun():
    # without a distributed environment, --gpus 2 starts two ranks itself
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps",
                        "1", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True,
                       timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2


def test_all_core_oracle_baseline():
    sys.path.insert(0, ROOT)
    import bench
    res = bench.cpu_all_cores(dict(bench.PARAMS), 2, budget_s=0.5)
    assert res["cores"] == 2 and res["value"] > 0 and "2 processes" in res["sample"]


def test_capture_digest_ignores_comments_only():
    sys.path.insert(0, ROOT)
    import bench
    code = "int f(int a) {\n    return a + 1;  // next\n}\n"
    commented = "/* header\n   text */\nint f(int a) {\n\n    return a + 1;  // other words\n}\n"
    changed = "int f(int a) {\n    return a + 2;  // next\n}\n"
    assert bench.code_digest([code]) == bench.code_digest([commented])
    assert bench.code_digest([code]) != bench.code_digest([changed])
    assert len(bench.kernel_source_digest()) == 16


if __name__ == "__main__":
    sys.exit(pytest.main([__file__, "-q"]))
