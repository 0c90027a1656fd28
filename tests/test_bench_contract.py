"""The bench's output contract, checked on the CPU.

The reference arm (the oracle's BiCGStab timed on the host cores) prints exactly one JSON
line with the keys the throughput line carries; under two ranks only rank 0 prints and
rank 1 exits 0 without work; the CUDA arm on a machine without a GPU exits non-zero and
prints no line, since nothing in it falls back to the CPU.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"}


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def json_lines(text):
    return [json.loads(x) for x in text.splitlines() if x.startswith("{")]


def test_reference_arm_prints_one_line():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "tiny_4x8"],
                  {"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert KEYS <= set(d), KEYS - set(d)
    assert d["impl"] == "reference" and d["unit"] == "sources/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["config"]["workload"] == "tiny_4x8"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_rank1_exits_without_work():
    r = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--workload", "tiny_4x8"],
                  {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert json_lines(r.stdout) == []


def test_cuda_arm_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = run_bench(["--steps", "1", "--warmup", "0", "--workload", "tiny_4x8", "--no-cpu-baseline"],
                  {"RANK": "0", "WORLD_SIZE": "1"})
    assert r.returncode != 0
    assert json_lines(r.stdout) == []


def test_stencil_traffic_comes_from_the_current_kernel_profile():
    """The bench's roofline.traffic is the committed ncu summary's DRAM bytes over algorithmic
    bytes for the current stencil version; the profile must exist, name that version, and give a
    ratio at least 1 (DRAM cannot move less than the kernel's compulsory bytes) for the default
    workload and for its N_v = 112 variant (the stencil does not depend on N_v)."""
    sys.path.insert(0, ROOT)
    import bench
    for wl in ("paper_24x128", "paper_24x128_nv112"):
        r = bench.measured_traffic_ratio(wl, "dslash_fp32")
        assert r is not None and 1.0 <= r < 3.0, (wl, r)
    assert bench.measured_traffic_ratio("medium_16x32", "dslash_fp32") is None   # taken on another version
