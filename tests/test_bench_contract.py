"""The benchmark's reference arm (the oracle on the host cores) prints one
JSON line with the contract's keys; runs on CPU in about a second."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "events/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1 and d["ms_per_step"] > 0
    assert d["config"]["workload"] and d["data"] == "synthetic"
    # the same config as the GPU arm's line (the headline workload)
    assert d["config"] == bench.headline_config(bench.N_EVENTS, 1)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_issue_roofline_from_counters(monkeypatch):
    # the issue roofline the bench prints for a form with committed counters
    # (device properties faked: no GPU needed)
    sys.path.insert(0, ROOT)
    import types
    import torch
    import bench
    monkeypatch.setattr(bench, "profile_counters",
                        lambda: {"plain_f32": {"warp_instructions_per_event": 80.0, "capture": "ncu ..."}})
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: types.SimpleNamespace(multi_processor_count=152))
    r = bench.issue_roofline(10_000_000, 2.5, "plain_f32", 2070.0)
    assert r["bound"] == "issue" and r["unit"] == "warp instructions/s"
    assert abs(r["peak"] - 152 * 4 * 2070e6) < 1.0
    assert abs(r["achieved"] - 80.0 * 1e7 / 2.5e-3) < 1.0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert bench.issue_roofline(10_000_000, 2.5, "dense_f32", 2070.0) is None   # no counters for the form
    assert bench.issue_roofline(10_000_000, 2.5, "plain_f32", None) is None     # no sampled clock


def test_committed_counters_match_the_kernel_sources():
    # profiles/counters.json records per-event counters of the chain kernel
    # as built from the current sources (the bench drops them otherwise)
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "profiles", "counters.json")) as f:
        d = json.load(f)
    if d["kernel_source_sha"] != bench.kernel_source_sha():
        pytest.skip("profiles/counters.json was captured from other kernel sources (re-capture on a GPU)")
    for form in ("plain_f32", "calls_f32_21", "batched_bf16_21", "dense_f32", "dense_bf16"):
        c = d["forms"][form]
        assert c["warp_instructions_per_event"] > 0 and c["dram_bytes_per_event"] > 0 and "ncu" in c["capture"]
