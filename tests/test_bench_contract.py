"""The one-JSON-line contract of bench.py: the reference arm (the oracle on
the host cores) runs here on CPU; the GPU arm's line is checked on a B300."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config"}


def _line(args, timeout):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                       text=True, timeout=timeout)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _line(["--impl", "reference", "--steps", "1", "--warmup", "0"], timeout=600)
    assert BASE_KEYS <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("config3")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.gpu
def test_gpu_arm_line():
    """the default line: config 3 headline, batched config 4 and served
    config 5 beside it (short settings), all rates in unique events"""
    d = _line(["--steps", "3", "--warmup", "3", "--cpu-seconds", "1", "--batch-steps", "1", "--plain-subset", "4",
               "--served-window", "1", "--served-plain", "2", "--served-spec-window", "0.5"], timeout=1800)
    assert BASE_KEYS <= set(d) and d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "events/s" and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("config3") and "l2" in d["config"]
    rf = d["roofline"]
    assert rf["bound"] in ("hbm", "tensor", "alu") and rf["peak"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9 and "measured on this GPU" in rf["peak_source"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    lb = d["latency_bound"]
    hw = lb["hw_floor"]
    assert 0 < hw["ns_per_event"] < lb["lone_lineage_ns_per_event"]
    if "longest_descent_events" in lb:
        assert lb["critical_events_per_step"] >= lb["longest_descent_events"]
        assert 0 < hw["frac_of_longest_floor"] < 1
    b = d["batched"]
    assert b["value"] > 0 and b["unit"] == "unique events/s" and b["speedup_vs_plain"] > 0
    bf = b["latency_bound"]["hw_floor"]
    assert b["latency_bound"]["critical_events_per_batch"] >= bf["longest_descent_events"]
    assert 0 < bf["frac_of_longest_floor"] < 1 and b["chain_floor_frac"] == bf["frac_of_longest_floor"]
    for key in ("served", "served_at_50_per_s"):
        s = d[key]
        assert s["requests"] > 0 and s["latency_s"]["p50"] > 0 and s["achieved_rate_per_s"] > 0
