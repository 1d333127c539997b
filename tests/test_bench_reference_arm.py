"""bench.py's reference arm (the oracle on the host cores, no GPU needed): one JSON
line with the headline's metric, unit and workload, its bounded sample described,
and under torchrun with two ranks (gloo) exactly one line, from rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lines(out):
    return [json.loads(ln) for ln in out.splitlines() if ln.startswith("{")]


def _check(line):
    sys.path.insert(0, ROOT)
    import bench
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"]["workload"] == "encmodel32-n32768"
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_one_process():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1, r.stdout
    _check(lines[0])
    assert lines[0]["n_gpus"] == 1


def test_reference_arm_two_ranks_prints_once():
    if torch.cuda.is_available():
        pytest.skip("host-side test (gloo); GPUs present")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = _lines(r.stdout)
    assert len(lines) == 1, r.stdout
    _check(lines[0])
    assert lines[0]["n_gpus"] == 2


def test_direct_oracle_timing_small_workload():
    """The directly timed oracle leg (whole inference of one query ciphertext) on the smallest
    workload: every query's labels equal the plaintext walk."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.oracle_direct("toy-n1024")
    assert r["labels_ok"] and r["queries"] == 32 and r["value"] > 0 and r["cores"] >= 1


def test_step_roofline_sums_families_at_their_binding_roofs():
    sys.path.insert(0, ROOT)
    import bench
    kernels = {"a": {"ms_per_step": 100.0, "hbm_frac": 0.2, "int_frac": 0.5},   # integer-bound: 50 ms at its roof
               "b": {"ms_per_step": 40.0, "hbm_frac": 0.75},                  # HBM-bound: 30 ms
               "c": {"ms_per_step": 10.0, "hbm_frac": 1.3}}                   # above its roof: counted at 10 ms
    r = bench.step_roofline(kernels, 200.0)
    assert abs(r["ms_at_roofs"] - 90.0) < 1e-9 and abs(r["frac"] - 0.45) < 1e-12
    assert bench.step_roofline({}, 200.0) is None and bench.step_roofline(None, 200.0) is None
