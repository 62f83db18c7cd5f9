"""Host logic of bench.py that runs without a GPU: the byte models behind the
roofline fractions, the traffic lookup, and the reference arm (the FP64 oracle timed
on the host) with the JSON line it prints."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_byte_models():
    # every stored value read once and written once per node and step
    assert bench.bytes_per_node("fp32") == 2 * 19 * 2 * 4 == 304
    assert bench.bytes_per_node("fp16") == bench.bytes_per_node("bf16") == 152
    assert bench.bytes_per_node("fp32_q5") == 2 * (19 + 5) * 4 == 192


def test_traffic_lookup_is_keyed_by_the_kernel_sources():
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    for st in ("fp32", "fp16", "fp32_q5"):
        t = bench.measured_traffic(st)
        assert t is None or t > 0.5 * bench.bytes_per_node(st) * 256 * 128 * 64
    assert bench.measured_traffic("no-such-storage") is None


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GLUPS" and d["value"] > 0
    assert d["metric"] == bench.METRIC and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["nodes"] == 256 * 128 * 64


def test_reduced_form_with_shan_chen_is_refused_on_the_command_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--storage", "fp32_q5",
                        "--model", "shan_chen"], capture_output=True, text=True, timeout=120,
                       cwd=ROOT)
    assert r.returncode != 0 and "colour-gradient" in r.stderr
