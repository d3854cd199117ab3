"""The benchmark's host-side accounting and its reference arm (the CPU oracle),
without a GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_series_bytes_per_site_by_hand():
    # K = 3: conversion of w_0 (16 + 8), sweep 1 (x 8, w_1 8, psi 16, acc 16, V 4),
    # last sweep (x 8, y_in 8, V 4, acc 16, psi 16)
    assert bench.series_bytes_per_site(3) == 24 + 52 + 52
    # K = 5 adds sweeps j = 2 and 3 (28 each; the accumulator waits for the last sweep)
    assert bench.series_bytes_per_site(5) == 24 + 52 + 52 + 28 + 28
    # K = 6 adds sweep j = 4, which adds terms 2, 3, 4 to the accumulator (28 + 32)
    assert bench.series_bytes_per_site(6) == 24 + 52 + 52 + 28 + 28 + 60
    # the graphene workload's 20 terms (17 middle sweeps, five of them touch the
    # accumulator: j = 4, 7, 10, 13, 16), stored and regenerated potential
    assert bench.series_bytes_per_site(20) == 24 + 2 * 52 + 17 * 28 + 5 * 32 == 764.0
    assert bench.series_bytes_per_site(20, 0.0) == 764.0 - 19 * 4
    with pytest.raises(ValueError):
        bench.series_bytes_per_site(2)


def test_reference_arm_prints_one_contract_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "0", "--dims", "24", "24", "4", "--R", "2"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["sample"]
    # the oracle runs on every host core, and the line says which CPU that was
    assert cb["cores"] == bench.host_cores() and cb["cpu_model"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["dims"] == [24, 24, 4] and d["config"]["R"] == 2
