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
    assert bench.bytes_per_node("fp16_q5") == 2 * (19 * 2 + 5 * 4) == 116


def test_traffic_lookup_is_keyed_by_the_kernel_sources():
    h = bench.kernel_source_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    n = 512 ** 3
    for st in ("fp32", "fp16", "fp32_q5"):
        t = bench.measured_traffic(st, "emulsion", n)
        assert t is None or t > 0.5 * bench.bytes_per_node(st) * n
    assert bench.measured_traffic("no-such-storage") is None


def test_traffic_of_a_smaller_capture_scales_per_node(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.kernel_source_hash()
    (prof / "traffic.txt").write_text(f"# comment\n{h} fp32 emulsion 1000 320000\n"
                                      f"0000000000000000 fp16 emulsion 1000 1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.measured_traffic("fp32", "emulsion", 10 ** 6) == 320.0 * 10 ** 6
    assert bench.measured_traffic("fp32", "emulsion") == 320000.0
    assert bench.measured_traffic("fp16", "emulsion", 10) is None       # other sources
    assert bench.measured_traffic("fp32", "channel", 10) is None


def test_clock_summary_and_gpu_selection():
    s = ["1965, 2070, 800.5, Not Active, Not Active, Not Active, Active",
         "2070, 2070, 900.0, Not Active, Not Active, Not Active, Not Active",
         "bad line"]
    rows = [r for r in (bench.parse_clock_line(x) for x in s) if r]
    d = bench.summarise_clocks(rows)
    assert d["sm_mhz"] == (1965 + 2070) / 2 and d["sm_max_mhz"] == 2070
    assert d["reasons"] == ["sw_power_cap"] and d["samples"] == 2
    assert bench.summarise_clocks([])["reasons"] == ["unsampled"]
    listing = "GPU-aaaa-1111, 0\nGPU-bbbb-2222, 1\n"
    # a torch UUID (without the GPU- prefix) selects that GPU whatever its local index
    assert bench.match_gpu("bbbb-2222", listing, 0) == "GPU-bbbb-2222"
    assert bench.match_gpu("GPU-AAAA-1111", listing, 1) == "GPU-aaaa-1111"
    assert bench.match_gpu("cccc", listing, 3) == "3" and bench.match_gpu(None, listing, 2) == "2"


def test_cpu_sample_is_a_box_of_the_initial_fields():
    import numpy as np
    from paper_2005_12764_gb300 import inputs
    rr, rb = inputs.paint_droplets((80, 300, 260), [(100.0, 120.0, 30.0, 10.0)])
    w = inputs.Workload("t", (80, 300, 260), rr, rb, {})
    a, b, shape, what = bench.cpu_sample(w, "emulsion")
    assert shape == bench.CPU_SAMPLE["emulsion"] and a.shape == shape and b.shape == shape
    nz, ny, nx = shape
    assert np.array_equal(a, rr[:nz, :ny, :nx]) and "periodic" in what
    assert bench.cpu_sample(w, "channel")[2] == w.shape


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "channel", "--steps", "1", "--warmup", "3"],
                       capture_output=True, text=True,
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
    assert d["cpu_baseline"]["sample"].startswith("1 steps of the whole lattice")


def test_reduced_form_with_shan_chen_is_refused_on_the_command_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--storage", "fp32_q5",
                        "--model", "shan_chen"], capture_output=True, text=True, timeout=120,
                       cwd=ROOT)
    assert r.returncode != 0 and "colour-gradient" in r.stderr


def test_near_contact_work_model():
    # the near-contact roofline: nodes with a ray counted like the oracle's gradient
    # threshold, the flop model and the FP32 peak from unit counts and clock
    import numpy as np
    import torch
    import oracle
    from paper_2005_12764_gb300 import inputs
    shape = (12, 16, 20)
    rr, rb = inputs.paint_droplets(shape, [(8.0, 8.0, 6.0, 4.0), (15.0, 6.0, 6.0, 3.5)])
    phi = (rr - rb) / (rr + rb)
    G = oracle.gradient(oracle.make_params(20, 16, 12), phi)
    want = int((np.sqrt((G ** 2).sum(axis=0)) >= 1e-3).sum())
    assert bench.listed_nodes_periodic(torch.from_numpy(phi)) == want > 0
    assert bench.nc_flops(100, 10, 19) == 100 * 45 + 10 * (19 * 27 + 20)
    assert abs(bench.fp32_peak_tflops(2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
