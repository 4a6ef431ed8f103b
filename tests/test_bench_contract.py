"""bench.py's CPU-side contract: argument parsing, the reference arm (the
oracle on the host cores, no GPU needed) and its one JSON line with the keys
the measurement contract names, and the O(N log N) CPU baseline helper."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout=300):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                       capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_help_lists_every_workload():
    out = _run(["--help"])
    for w in ("ckks_hmul_n65536", "mixed_batch", "tfhe_blind_rotation", "tfhe_cmux", "ckks_bconv",
              "ckks_rescale", "natural_order", "otf_twiddles", "word32", "n_sweep", "cost_model", "serving"):
        assert w in out, w


def test_reference_arm_line():
    line = json.loads(_run(["--impl", "reference", "--steps", "1", "--warmup", "0"]).strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["workload"] == "ckks_hmul_n65536"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["cpu"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_radix2_baseline_helper():
    sys.path.insert(0, ROOT)
    import bench
    value, cores, seconds = bench.radix2_sample()
    assert value > 0 and cores >= 1 and seconds > 0
