"""Benchmark of the fused colour-gradient LB step on GB300.

Default workload: the dense emulsion, 512^3 periodic D3Q19 nodes (134,217,728) with
random non-overlapping droplets at volume fraction 0.35 (radii 6-12, seeded random
sequential addition), Kolmogorov forcing F_x = 1e-5 sin(2 pi y / 512), near-contact
force A = 0.01 within 3 lu, sigma = 0.01, beta = 0.7, tau = 1, FP32 storage. One step =
one lattice update of every node (the near-contact pass and the fused step kernel).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload emulsion|channel]
                  [--storage fp32|fp16|bf16|fp32_q5|fp16_q5] [--impl ours|reference]
                  [--model colour|shan_chen] [--no-serving] [--no-models] [--no-cpu-baseline]

Prints one JSON line. ``value`` is GLUPS (10^9 lattice-node updates per second) over
all ranks, device-resident; the timed K-step loop is repeated until about a second
has been timed (so that the clock sampler sees it) and the median repeat is
reported. ``e2e`` times the same job through the public C-ABI with host buffers
(set fields from pinned host memory, K steps, fields back to the host);
``roofline`` relates the step kernel's algorithmic bytes (2 x 19 x 2 populations per
node, read once and written once) to the measured HBM bandwidth; ``fp16_store``
repeats the device-resident measurement on the same lattice with FP16 deviation
storage (and, inside it, BF16), ``fp32_q5_store`` with the reduced FP32 form (19
totals and 5 recolouring coefficients per node), ``fp16_q5_store`` with its FP16
variant (FP16 totals, exact coefficients); ``gel_640`` times the bicontinuous
gel quench (640^3, tau = 0.8, 2 % pinning sites, near contact on, FP32) with the
near-contact pass's share; ``channel`` the microfluidic-crystal channel (256 x 128
x 64); ``shan_chen`` and ``sheared_bijel`` the Shan-Chen model on the channel and the
sheared-bijel channel with sliding walls; ``serving`` runs the served request stream
(256 droplet / sheared-droplet runs of edge 32-128, Poisson arrivals at 50/s, FP16
storage) through the serving engine and reports p50/p99 latency beside aggregate
GLUPS; ``cpu_baseline`` times the FP64 oracle on the host cores (all, and one) on a
bounded sample of the workload. ``--impl reference`` times the oracle itself on that
sample (the method has no other reference implementation). Multi-GPU runs are
independent replicas: one lattice per rank, the request stream sharded over the
ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS & % HBM roofline, FP32 vs FP16-store; served-run p50/p99 latency"
Q, C = 19, 2

WORKLOADS = {
    "emulsion": "dense emulsion 512^3 periodic, volume fraction 0.35, radii 6-12, "
                "Kolmogorov F_x = 1e-5 sin(2 pi y/512), NC on (A = 0.01, h_min = 3)",
    "channel": "microfluidic-crystal channel 256x128x64, 40 droplets, walls y/z, NC on",
    "channel_sc": "microfluidic-crystal channel 256x128x64, 40 droplets, walls y/z, "
                  "Shan-Chen G_sc = 1.6",
}

# Bounded sample of a workload for the oracle (CPU baseline, reference arm): a box of
# the workload's initial fields, stepped as a periodic lattice of its own with the
# workload's parameters. (nz, ny, nx) of the box.
CPU_SAMPLE = {"emulsion": (64, 256, 256), "channel": None, "channel_sc": None}

KERNEL_SOURCES = ("lbm_step.cu", "lbm_device.cuh")   # what the step kernel is built from


def kernel_source_hash() -> str:
    d = os.path.join(ROOT, "paper_2005_12764_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def bytes_per_node(storage: str) -> int:
    """Algorithmic HBM bytes of one node and step: every stored value read once and
    written once (2 x 2Q values; in the reduced forms 2 x (Q totals + 5 FP32
    coefficients), the totals FP32 or FP16)."""
    if storage == "fp32_q5":
        return 2 * (Q + 5) * 4
    if storage == "fp16_q5":
        return 2 * (Q * 2 + 5 * 4)
    return 2 * Q * C * (4 if storage == "fp32" else 2)


# Algorithmic FP32 work of the near-contact pass (Eq. 11 as read: a film measured along
# -G'/|G'| by trilinear samples of the lagged colour field), in flops:
NC_FLOPS_NODE = 45     # the lagged gradient G' (18 multiply-adds) and |G'|, the unit ray
NC_FLOPS_SAMPLE = 27   # a sample: t n' (3 mul), the cell fractions (3 sub), 7 lerps x 3
NC_FLOPS_RAY = 20      # the two crossings (linear interpolation) and A_h[h]
FP32_LANES_PER_SM = 128


def nc_flops(nodes: int, listed: int, nsamp: int) -> int:
    """Flops of one near-contact pass: every node's gradient, and every listed node's
    ray (|G'| >= 1e-3) of nsamp samples with its two crossings."""
    return nodes * NC_FLOPS_NODE + listed * (nsamp * NC_FLOPS_SAMPLE + NC_FLOPS_RAY)


def fp32_peak_tflops(sm_mhz: float, sms: int = 152) -> float:
    """FP32 (non-tensor) peak: SMs x FP32 lanes x 2 flops (a multiply-add) x clock."""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def listed_nodes_periodic(phi, g_min: float = 1e-3) -> int:
    """Nodes of a periodic lattice whose isotropic colour gradient (3 w_i = 1/6 faces,
    1/12 edges) has |G| >= g_min: those the near-contact pass gives a ray (a torch
    tensor [nz, ny, nx], on any device)."""
    import torch
    G = [torch.zeros_like(phi) for _ in range(3)]
    for cz in (-1, 0, 1):
        for cy in (-1, 0, 1):
            for cx in (-1, 0, 1):
                n = abs(cx) + abs(cy) + abs(cz)
                if n == 0 or n == 3:
                    continue
                w3 = 1.0 / 6.0 if n == 1 else 1.0 / 12.0
                v = torch.roll(phi, shifts=(-cz, -cy, -cx), dims=(0, 1, 2))
                for a, c in enumerate((cx, cy, cz)):
                    if c:
                        G[a] += (w3 * c) * v
    return int(((G[0] ** 2 + G[1] ** 2 + G[2] ** 2).sqrt() >= g_min).sum().item())


def measured_traffic(storage: str, workload: str = "emulsion", nodes: int | None = None):
    """DRAM bytes per launch of the step kernel on `workload` from the committed ncu
    summary, if it was taken on the current kernel sources; else None. A line taken on
    a smaller case of the workload gives bytes per node, scaled to `nodes`."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if line.startswith("#") or len(parts) < 5:
            continue
        h, st, wl, captured_nodes, b = parts[:5]
        if h == want and st == storage and wl == workload:
            per_node = float(b) / float(captured_nodes)
            return per_node * (nodes if nodes is not None else float(captured_nodes))
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def match_gpu(uuid: str | None, smi_listing: str, local: int) -> str:
    """nvidia-smi's -i argument for a torch device: the UUID nvidia-smi lists for it
    (`smi_listing` = lines "uuid, index" of `nvidia-smi --query-gpu=uuid,index`), since
    nvidia-smi ignores CUDA_VISIBLE_DEVICES and a local index may name another GPU;
    the local index when the UUID is unknown or not listed."""
    if uuid:
        u = uuid.lower().removeprefix("gpu-")
        for ln in smi_listing.splitlines():
            parts = [p.strip() for p in ln.split(",")]
            if parts and parts[0].lower().removeprefix("gpu-") == u:
                return parts[0]
    return str(local)


def gpu_selector(local: int) -> str:
    try:
        import torch
        u = getattr(torch.cuda.get_device_properties(local), "uuid", None)
        r = subprocess.run(["nvidia-smi", "--query-gpu=uuid,index", "--format=csv,noheader"],
                           capture_output=True, text=True, timeout=10)
        return match_gpu(str(u) if u is not None else None, r.stdout, local)
    except Exception:
        return str(local)


CLOCK_FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                "clocks_event_reasons.sw_power_cap")
REASON_NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


def parse_clock_line(line: str):
    parts = [p.strip() for p in line.split(",")]
    return parts if len(parts) >= 7 else None


def summarise_clocks(samples):
    """Median SM clock, maximum clock and the throttle reasons seen in nvidia-smi
    samples (lists of the CLOCK_FIELDS columns)."""
    if not samples:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

    def num(s):
        try:
            return float(s)
        except ValueError:
            return None
    sm = [v for v in (num(s[0]) for s in samples) if v is not None]
    mx = [v for v in (num(s[1]) for s in samples) if v is not None]
    reasons = sorted({REASON_NAMES[k] for s in samples for k in range(4)
                      if s[3 + k].lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
            "samples": len(samples)}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons of one GPU, sampled every 100 ms in a
    thread, plus one query at entry and one at exit (so a short region still has a
    record)."""

    def __init__(self, selector):
        self.sel = selector
        self.samples = []
        self.edges = []
        self.proc = None

    def _query_once(self):
        try:
            r = subprocess.run(["nvidia-smi", "-i", self.sel, f"--query-gpu={CLOCK_FIELDS}",
                                "--format=csv,noheader,nounits"], capture_output=True,
                               text=True, timeout=10)
            s = parse_clock_line(r.stdout.strip().splitlines()[0]) if r.stdout.strip() else None
            if s:
                self.edges.append(s)
        except (FileNotFoundError, OSError, subprocess.TimeoutExpired, IndexError):
            pass

    def __enter__(self):
        self._query_once()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.sel, f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            s = parse_clock_line(line)
            if s:
                self.samples.append(s)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self._query_once()

    def summary(self):
        d = summarise_clocks(self.samples if self.samples else self.edges)
        d["source"] = "100 ms samples" if self.samples else "queries at entry and exit"
        d["gpu"] = self.sel
        return d


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_key(args):
    if args.model == "shan_chen":
        return "channel_sc"
    return args.workload


def make_workload(key, size=512):
    from paper_2005_12764_gb300 import inputs
    if key == "emulsion":
        return inputs.dense_emulsion(L=size)
    if key == "channel_sc":
        return inputs.channel_shan_chen()
    return inputs.channel_droplets()


def host_cpu():
    """Host CPU model (lscpu) and core count."""
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for ln in r.stdout.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (FileNotFoundError, OSError, subprocess.TimeoutExpired):
        pass
    return {"model": model, "cores": os.cpu_count()}


def cpu_sample(w, key):
    """Fields and shape of the oracle's bounded sample of workload w: the whole
    lattice, or a box of its initial fields (CPU_SAMPLE) stepped as a periodic lattice
    with the workload's parameters."""
    box = CPU_SAMPLE.get(key)
    if box is None:
        return w.rho_r, w.rho_b, w.shape, "the whole lattice"
    nz, ny, nx = box
    rr = w.rho_r[:nz, :ny, :nx].copy()
    rb = w.rho_b[:nz, :ny, :nx].copy()
    return rr, rb, box, f"a {nx}x{ny}x{nz} box of its initial fields, periodic"


def oracle_rate(rr, rb, shape, params, steps, warm=1):
    """Oracle lattice updates per second on this host over `steps` steps."""
    import oracle
    nz, ny, nx = shape
    lat = oracle.Lattice(oracle.make_params(nx, ny, nz, **params))
    lat.set_fields(rr, rb)
    lat.step(warm)
    t0 = time.perf_counter()
    lat.step(steps)
    dt = time.perf_counter() - t0
    lat.close()
    return nx * ny * nz * steps / dt, dt


def one_core_rate(key, steps):
    """The oracle on one core: a child process with OMP_NUM_THREADS=1 (the OpenMP
    runtime of this process already has its thread count)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-rate-only",
                        "--workload", key, "--cpu-steps", str(steps)], capture_output=True,
                       text=True, env=env, timeout=900)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_rate_only(args):
    key = workload_key(args)
    w = make_workload(key)
    rr, rb, shape, what = cpu_sample(w, key)
    rate, dt = oracle_rate(rr, rb, shape, w.params, args.cpu_steps)
    print(json.dumps({"rate": rate, "dt": dt, "sample": what}), flush=True)


def run_reference(args):
    """The FP64 oracle timed on the host cores, on the same workload and metric (each
    step on the bounded sample of the workload)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    key = workload_key(args)
    w = make_workload(key)
    rr, rb, shape, what = cpu_sample(w, key)
    import oracle
    nz, ny, nx = shape
    lat = oracle.Lattice(oracle.make_params(nx, ny, nz, **w.params))
    lat.set_fields(rr, rb)
    lat.step(args.warmup)
    t0 = time.perf_counter()
    lat.step(args.steps)
    dt = time.perf_counter() - t0
    n = nx * ny * nz
    glups = n * args.steps / dt / 1e9
    cpu = host_cpu()
    line = {"impl": "reference", "metric": METRIC, "value": glups, "unit": "GLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[key], "nodes": w.rho_r.size,
                       "storage": "f64 (oracle)"},
            "cpu_baseline": {"value": glups, "unit": "GLUPS", "cores": cpu["cores"],
                             "cpu": cpu["model"], "kind": "oracle",
                             "sample": f"{args.steps} steps of {what} ({n} nodes)"},
            "e2e": {"value": glups, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_steps(lat, stream, steps, min_total_s=1.0, max_reps=20):
    """Per-repeat milliseconds of `steps` steps queued back to back (CUDA events on the
    library's stream, synchronised on both sides), repeated until about min_total_s
    has been timed."""
    import torch
    reps = []
    total = 0.0
    while len(reps) < max_reps and (total < min_total_s * 1e3 or len(reps) < 1):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lat.step(steps)
        b.record(stream)
        stream.synchronize()
        ms = a.elapsed_time(b)
        reps.append(ms)
        total += ms
    return reps


def device_resident(lbm, w, storage, steps, warmup, stream, local, pins=None, inplace=0):
    """GLUPS of `steps` steps queued back to back (median repeat), the mean step-kernel
    and near-contact pass times (ms, the library's own events; in place, the step
    kernel time covers the colour-field and collide passes), and the lattice's
    species-mass drift over the run."""
    import torch
    nz, ny, nx = w.shape
    lat = lbm.Lattice(lbm.make_params(nx, ny, nz, storage=storage, stream=stream.cuda_stream,
                                      inplace=inplace, **w.params))
    lat.set_fields(torch.from_numpy(w.rho_r).to(f"cuda:{local}"),
                   torch.from_numpy(w.rho_b).to(f"cuda:{local}"))
    if pins is not None:
        lat.set_pin_mask(torch.from_numpy(pins).to(f"cuda:{local}"))
    m0 = lat.observables()[:2]
    lat.step(warmup)
    lat.sync()
    reps = timed_steps(lat, stream, steps, min_total_s=0.5, max_reps=5)
    ms = statistics.median(reps)
    kt = max(5, min(steps, 20))
    nc_ms, step_ms, _ = lat.step_timed(kt)
    m1 = lat.observables()[:2]
    taken = lat.steps_taken
    lat.close()
    drift = [abs(float(m1[k]) - float(m0[k])) / float(m0[k]) for k in range(2)]
    return {"value": nx * ny * nz * steps / (ms * 1e-3) / 1e9, "ms_per_step": ms / steps,
            "kernel_ms": step_ms / kt, "near_contact_pass_ms": nc_ms / kt,
            "mass_drift_rel": {"red": drift[0], "blue": drift[1], "steps": taken}}


def serving_run(lbm, rank, world, dist, local):
    """The served request stream (sharded over replicas) through the serving engine."""
    from paper_2005_12764_gb300 import inputs, replicas, serving
    reqs = replicas.shard(inputs.serving_requests(), rank, world)
    # shortest job first over 16 resident lattices: the stream is saturated (about five
    # times more work arrives per second than one GPU completes), so the median
    # latency is set by the admission order
    eng = lbm.Engine(budget_bytes=64 << 30, max_slots=16, chunk_steps=50, policy="sjf")
    rep = serving.serve(eng, reqs, storage="fp16")
    eng.close()
    lat = replicas.gather_lists(rep["latency_s"], dist)
    wall = replicas.max_over_ranks(rep["wall_s"], dist, f"cuda:{local}")
    lups = replicas.sum_over_ranks(rep["lattice_updates"], dist, f"cuda:{local}")
    first = min(r["arrival_s"] for r in inputs.serving_requests())
    return {"requests": len(lat), "storage": "fp16", "policy": "shortest job first, 16 slots",
            "p50_ms": serving.percentile(lat, 50) * 1e3,
            "p99_ms": serving.percentile(lat, 99) * 1e3,
            "glups": lups / (wall - first) / 1e9, "wall_s": wall,
            "stream": "256 requests, edge {32,48,64,96,128}, R = L/4, sigma U[0.005,0.03], "
                      "steps U[200,2000], half sheared (Kolmogorov 1e-5), Poisson 50/s",
            "engine": {k: rep["engine"][k] for k in ("ticks", "peak_bytes", "planes_per_cta")}}


def other_workloads(lbm, stream, local, key, steps=20, warmup=5):
    """Device-resident GLUPS of more workloads of the same step: the gel quench at
    640^3 (FP32), the channel (when it is not the timed workload), the Shan-Chen model
    on the channel geometry, and the sheared-bijel channel (1024 x 128 x 128, sliding
    walls, near contact on) after 300 steps of coarsening from the quench."""
    import torch
    from paper_2005_12764_gb300 import inputs
    out = {}
    hbm = peaks()[0]

    def frac(kernel_ms, nodes, storage="fp32"):
        return bytes_per_node(storage) * nodes / (kernel_ms * 1e-3) / 1e9 / hbm

    # the bicontinuous gel quench, 640^3, FP32 (two copies, 81 GB)
    g = inputs.bicontinuous()
    n = g.rho_r.size
    d = device_resident(lbm, g, "fp32", steps, warmup, stream, local, pins=g.pins)
    d.update({"workload": "bicontinuous gel quench 640^3 periodic, phi0 U(+-0.01), 2 % pins, "
                          "tau = 0.8, sigma = 0.015, A_nc = 0.02, FP32, steps "
                          f"{warmup + 1}-{warmup + steps} after the quench",
              "unit": "GLUPS", "nodes": n,
              "roofline_frac": frac(d["kernel_ms"], n),
              "near_contact_share": d["near_contact_pass_ms"] / d["ms_per_step"]})
    out["gel_640"] = d
    # the same quench with FP16 deviation storage, two copies (39.8 GB) and in place
    # (one copy, 19.9 GB: two passes per step, the populations read twice)
    for tag, inplace in (("gel_640_fp16", 0), ("gel_640_fp16_inplace", 1)):
        d = device_resident(lbm, g, "fp16", steps, warmup, stream, local, pins=g.pins,
                            inplace=inplace)
        d.update({"workload": "bicontinuous gel quench 640^3 as above, FP16 deviation storage"
                              + (", in place (one population copy)" if inplace else ""),
                  "unit": "GLUPS", "nodes": n,
                  "roofline_frac": frac(d["kernel_ms"], n, "fp16"),
                  "pass_bytes_per_node": bytes_per_node("fp16") * (3 if inplace else 2) // 2,
                  "near_contact_share": d["near_contact_pass_ms"] / d["ms_per_step"]})
        out[tag] = d
    del g
    if key != "channel":
        w = inputs.channel_droplets()
        n = w.rho_r.size
        d = device_resident(lbm, w, "fp32", 200, 10, stream, local)
        d.update({"workload": WORKLOADS["channel"], "unit": "GLUPS", "nodes": n,
                  "roofline_frac": frac(d["kernel_ms"], n),
                  "traffic": measured_traffic("fp32", "channel", n)})
        out["channel"] = d

    def timed(lat, k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lat.step(k)
        b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b) / k

    w = inputs.channel_shan_chen()
    nz, ny, nx = w.shape
    lat = lbm.Lattice(lbm.make_params(nx, ny, nz, stream=stream.cuda_stream, **w.params))
    lat.set_fields(w.rho_r, w.rho_b)
    lat.step(10)
    ms = timed(lat, 200)
    _, k_ms, _ = lat.step_timed(20)
    lat.close()
    alg = bytes_per_node("fp32") * nx * ny * nz
    out["shan_chen"] = {"workload": "channel 256x128x64, 40 droplets, walls y/z, G_sc = 1.6, FP32",
                        "value": nx * ny * nz / (ms * 1e-3) / 1e9, "unit": "GLUPS",
                        "ms_per_step": ms, "kernel_ms": k_ms / 20,
                        "roofline_frac": alg / (k_ms / 20 * 1e-3) / 1e9 / hbm,
                        "algorithmic_bytes_per_launch": alg}
    w = inputs.sheared_bijel()
    nz, ny, nx = w.shape
    lat = lbm.Lattice(lbm.make_params(nx, ny, nz, stream=stream.cuda_stream, **w.params))
    lat.set_fields(torch.from_numpy(w.rho_r).to(f"cuda:{local}"),
                   torch.from_numpy(w.rho_b).to(f"cuda:{local}"))
    lat.step(300)
    ms = timed(lat, 50)
    nc_ms, k_ms, _ = lat.step_timed(10)
    lat.close()
    out["sheared_bijel"] = {"workload": "1024x128x128, walls y (sliding +-0.01) and z, "
                                        "quench noise 0.01, NC on, FP32, after 300 steps",
                            "value": nx * ny * nz / (ms * 1e-3) / 1e9, "unit": "GLUPS",
                            "ms_per_step": ms, "kernel_ms": k_ms / 10,
                            "near_contact_pass_ms": nc_ms / 10}
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2005_12764_gb300 import build_lib, lbm, replicas

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build_lib.build()
    key = workload_key(args)
    w = make_workload(key, args.size)
    nz, ny, nx = w.shape
    N = nx * ny * nz
    stream = torch.cuda.Stream()
    P = lbm.make_params(nx, ny, nz, storage=args.storage, stream=stream.cuda_stream,
                        inplace=1 if args.inplace else 0, **w.params)
    lat = lbm.Lattice(P)
    dev_rr = torch.from_numpy(w.rho_r).to(f"cuda:{local}")
    dev_rb = torch.from_numpy(w.rho_b).to(f"cuda:{local}")
    torch.cuda.synchronize()
    lat.set_fields(dev_rr, dev_rb)
    del dev_rr, dev_rb
    lat.step(args.warmup)
    lat.sync()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timing: K steps queued back to back, CUDA events on the
    # stream the kernels run on; the K-step loop is repeated until about a second has
    # been timed (the clock sampler's 100 ms samples then cover it) and the median
    # repeat is taken
    barrier()
    with ClockSampler(gpu_selector(local)) as clk:
        reps = timed_steps(lat, stream, args.steps, min_total_s=1.0)
    barrier()
    med_ms = statistics.median(reps)
    total_ms = replicas.max_over_ranks(med_ms, dist if world > 1 else None, f"cuda:{local}")
    ms_per_step = total_ms / args.steps
    glups = world * N * args.steps / (total_ms * 1e-3) / 1e9
    # per-kernel durations (events around each launch, inside the library)
    kt = max(5, min(args.steps, 20))
    nc_ms, step_ms, _ = lat.step_timed(kt)
    kern_ms = step_ms / kt
    nc_avg_ms = nc_ms / kt
    # nodes the near-contact pass gives a ray, on the lagged field those steps read
    listed = None
    if w.params.get("A_nc", 0.0) > 0 and not (w.params.get("wall_y") or w.params.get("wall_z")):
        phi_dev = torch.empty(w.shape, dtype=torch.float64, device=f"cuda:{local}")
        lat.get_fields({"phi": phi_dev})
        listed = listed_nodes_periodic(phi_dev)
        del phi_dev
    # ---- end to end through the public API with pinned host buffers
    host_rr = torch.from_numpy(w.rho_r).pin_memory()
    host_rb = torch.from_numpy(w.rho_b).pin_memory()
    outs = {"rho_r": torch.empty(w.shape, dtype=torch.float64).pin_memory(),
            "rho_b": torch.empty(w.shape, dtype=torch.float64).pin_memory(),
            "u": torch.empty((3,) + w.shape, dtype=torch.float64).pin_memory(),
            "phi": torch.empty(w.shape, dtype=torch.float64).pin_memory()}
    barrier()
    t0 = time.perf_counter()
    lat.set_fields(host_rr, host_rb)
    lat.step(args.steps)
    lat.get_fields(outs)
    e2e_s = replicas.max_over_ranks(time.perf_counter() - t0, dist if world > 1 else None,
                                    f"cuda:{local}")
    e2e = world * N * args.steps / e2e_s / 1e9
    h2d = 2 * N * 8
    d2h = 6 * N * 8
    del host_rr, host_rb, outs

    # ---- roofline of the step kernel
    alg_bytes = bytes_per_node(args.storage) * N
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    traffic = measured_traffic(args.storage, key, N)

    obs = lat.observables()
    finite = bool(np.isfinite(obs[:5]).all())
    launches = args.steps * lat.launches_per_step
    lat.close()
    # the same workload with FP16 / BF16 deviation storage and the reduced FP32 form
    # (device-resident, as `value`)
    fp16 = q5 = q5h = None
    if args.storage == "fp32" and not args.no_variants:
        d16 = device_resident(lbm, w, "fp16", args.steps, args.warmup, stream, local)
        d16["value"] = replicas.sum_over_ranks(d16["value"], dist if world > 1 else None,
                                               f"cuda:{local}")
        alg16 = bytes_per_node("fp16") * N
        d16.update({"unit": "GLUPS",
                    "roofline_frac": alg16 / (d16["kernel_ms"] * 1e-3) / 1e9 / peak,
                    "algorithmic_bytes_per_launch": alg16,
                    "traffic": measured_traffic("fp16", key, N)})
        fp16 = d16
        db = device_resident(lbm, w, "bf16", args.steps, args.warmup, stream, local)
        db["value"] = replicas.sum_over_ranks(db["value"], dist if world > 1 else None,
                                              f"cuda:{local}")
        db.update({"unit": "GLUPS",
                   "roofline_frac": alg16 / (db["kernel_ms"] * 1e-3) / 1e9 / peak})
        fp16["bf16"] = db
    if args.storage == "fp32" and args.model == "colour" and not args.no_variants:
        # the reduced FP32 form (Q + 5 values per node; colour-gradient states only),
        # against its own byte model of 192 bytes per node and step
        d5 = device_resident(lbm, w, "fp32_q5", args.steps, args.warmup, stream, local)
        d5["value"] = replicas.sum_over_ranks(d5["value"], dist if world > 1 else None,
                                              f"cuda:{local}")
        alg5 = bytes_per_node("fp32_q5") * N
        d5.update({"unit": "GLUPS",
                   "roofline_frac": alg5 / (d5["kernel_ms"] * 1e-3) / 1e9 / peak,
                   "algorithmic_bytes_per_launch": alg5,
                   "traffic": measured_traffic("fp32_q5", key, N)})
        q5 = d5
        # and its FP16 variant (FP16 totals, exact FP32 coefficients: 116 bytes per node)
        dh = device_resident(lbm, w, "fp16_q5", args.steps, args.warmup, stream, local)
        dh["value"] = replicas.sum_over_ranks(dh["value"], dist if world > 1 else None,
                                              f"cuda:{local}")
        algh = bytes_per_node("fp16_q5") * N
        dh.update({"unit": "GLUPS",
                   "roofline_frac": algh / (dh["kernel_ms"] * 1e-3) / 1e9 / peak,
                   "algorithmic_bytes_per_launch": algh,
                   "traffic": measured_traffic("fp16_q5", key, N)})
        q5h = dh
    others = None
    if not args.no_models:
        others = other_workloads(lbm, stream, local, key)
    serving_rep = None
    if not args.no_serving:
        serving_rep = serving_run(lbm, rank, world, dist if world > 1 else None, local)
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            rr, rb, shape, what = cpu_sample(w, key)
            n_s = shape[0] * shape[1] * shape[2]
            rate, dt = oracle_rate(rr, rb, shape, w.params, args.cpu_steps)
            hc = host_cpu()
            cpu = {"value": rate / 1e9, "unit": "GLUPS", "cores": hc["cores"], "cpu": hc["model"],
                   "kind": "oracle",
                   "sample": f"{args.cpu_steps} FP64 steps of {what} ({n_s} nodes, {dt:.1f} s)"}
            one = one_core_rate(key, max(1, args.cpu_steps // 10))
            if one:
                cpu["one_core"] = {"value": one["rate"] / 1e9, "unit": "GLUPS", "cores": 1,
                                   "sample": f"{max(1, args.cpu_steps // 10)} FP64 steps of "
                                             f"{one['sample']} ({one['dt']:.1f} s)"}
        line = {
            "metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[key] if args.size == 512 or key != "emulsion"
                       else WORKLOADS[key].replace("512", str(args.size)),
                       "nodes": N, "storage": args.storage,
                       "inplace": bool(args.inplace),
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (%.0f MB of populations per copy)"
                             % (bytes_per_node(args.storage) * N / 2 / 1e6),
                       "timed_repeats": len(reps),
                       "repeat_ms": [round(r, 3) for r in reps]},
            "e2e": {"value": e2e, "unit": "GLUPS",
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "job": "set_fields(host) + K steps + get_fields(host)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} HBM copy bandwidth",
                         "kernel": "step_kernel (fused stream/collide/perturb/recolour)",
                         "kernel_ms": kern_ms,
                         "near_contact_pass_ms": nc_avg_ms,
                         "ghost_fill": "written by the near-contact pass (no launch of its own)",
                         "algorithmic_bytes_per_launch": alg_bytes},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "finite": finite,
        }
        if listed is not None:
            # the near-contact pass takes most of the step on this workload; it is bound by
            # instruction issue and latency (ALU), not by HBM
            h_cut = w.params.get("h_cut") or 2.0 * w.params.get("h_min", 3.0)
            nsamp = int(math.floor(2.0 * (h_cut + 3.0))) + 1
            fl = nc_flops(N, listed, nsamp)
            mhz = line["clocks"].get("sm_max_mhz") or 2070.0
            ach = fl / (nc_avg_ms * 1e-3) / 1e12
            pk = fp32_peak_tflops(float(mhz))
            line["near_contact_roofline"] = {
                "bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
                "kernel": "nc_block_kernel (near-contact film measurement, with the ghost copies)",
                "kernel_ms": nc_avg_ms, "flops_per_launch": fl, "listed_fraction": listed / N,
                "samples_per_ray": nsamp,
                "peak_source": f"152 SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x {mhz} MHz"}
        if fp16:
            line["fp16_store"] = fp16
        if q5:
            line["fp32_q5_store"] = q5
        if q5h:
            line["fp16_q5_store"] = q5h
        if others:
            line.update(others)
        if serving_rep:
            line["serving"] = serving_rep
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_study(args):
    """The workloads' own long runs (not a bench line): `--study emulsion` runs the
    512^3 emulsion for `--study-steps` steps (2000) in every storage form and reports
    each form's species-mass drift and droplet census against FP32's; `--study gel`
    runs the 640^3 gel quench in FP32 and in the FP16 reduced form, reporting GLUPS and
    the peak of the structure factor S(k, t) every `--every` steps."""
    import numpy as np
    import torch

    from paper_2005_12764_gb300 import build_lib, inputs, lbm

    torch.cuda.set_device(0)
    build_lib.build()
    stream = torch.cuda.Stream()

    def lattice(w, storage, pins=None):
        nz, ny, nx = w.shape
        lat = lbm.Lattice(lbm.make_params(nx, ny, nz, storage=storage,
                                          stream=stream.cuda_stream, **w.params))
        lat.set_fields(torch.from_numpy(w.rho_r).cuda(), torch.from_numpy(w.rho_b).cuda())
        if pins is not None:
            lat.set_pin_mask(torch.from_numpy(pins).cuda())
        return lat

    def timed(lat, k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        lat.step(k)
        b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b)

    out = {"study": args.study, "steps": args.study_steps}
    if args.study == "emulsion":
        w = make_workload("emulsion", args.size)
        N = w.rho_r.size
        forms = {}
        for st in ("fp32", "fp16", "bf16", "fp32_q5", "fp16_q5"):
            lat = lattice(w, st)
            m0 = lat.observables()[:2]
            n0, s0 = lat.droplets()
            ms = timed(lat, args.study_steps)
            m1 = lat.observables()[:2]
            n1, s1 = lat.droplets()
            hist = np.bincount(np.minimum(np.round(np.cbrt(3 * s1 / (4 * np.pi))).astype(int), 40),
                               minlength=41)
            forms[st] = {"glups": N * args.study_steps / (ms * 1e-3) / 1e9,
                         "mass_drift_rel": [abs(float(m1[k] - m0[k])) / float(m0[k]) for k in range(2)],
                         "droplets_start": n0, "droplets_end": n1,
                         "radius_histogram_end": hist.tolist(),
                         "largest_end": [int(v) for v in s1[:3]]}
            lat.close()
        ref = forms["fp32"]["radius_histogram_end"]
        for st, d in forms.items():
            d["histogram_l1_vs_fp32"] = int(np.abs(np.array(d["radius_histogram_end"]) -
                                                   np.array(ref)).sum())
        out.update({"workload": WORKLOADS["emulsion"], "forms": forms})
    else:
        w = inputs.bicontinuous()
        N = w.rho_r.size
        runs = {}
        for st in ("fp32", "fp16_q5"):
            lat = lattice(w, st, w.pins)
            series, total_ms, done = [], 0.0, 0
            while done < args.study_steps:
                k = min(args.every, args.study_steps - done)
                total_ms += timed(lat, k)
                done += k
                kk, S, modes = lat.structure_factor(560)
                j = 1 + int(np.argmax(S[1:]))
                series.append({"step": done, "k_peak": float(kk[j]), "S_peak": float(S[j])})
            runs[st] = {"glups": N * done / (total_ms * 1e-3) / 1e9, "S_peak_vs_t": series}
            lat.close()
        out.update({"workload": "bicontinuous gel quench 640^3, 2 % pins, tau = 0.8", "runs": runs})
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="emulsion", choices=["emulsion", "channel"])
    ap.add_argument("--size", type=int, default=512,
                    help="edge of the emulsion box (smaller cases for profiler captures)")
    ap.add_argument("--storage", default="fp32",
                    choices=["fp32", "fp16", "bf16", "fp32_q5", "fp16_q5"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--inplace", action="store_true",
                    help="one population copy updated in place (kernel_ms then covers the "
                         "colour-field and collide passes)")
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP16/BF16 and reduced-form lines")
    ap.add_argument("--model", default="colour", choices=["colour", "shan_chen"],
                    help="model of the timed workload (shan_chen: the channel)")
    ap.add_argument("--no-models", action="store_true",
                    help="skip the gel, channel, Shan-Chen and sheared-bijel lines")
    ap.add_argument("--oracle-rate-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--study", choices=["emulsion", "gel"],
                    help="long run of a workload instead of the bench line")
    ap.add_argument("--study-steps", type=int, default=2000)
    ap.add_argument("--every", type=int, default=1000)
    args = ap.parse_args()
    if args.storage in ("fp32_q5", "fp16_q5") and args.model == "shan_chen":
        ap.error("the reduced storage form holds colour-gradient states only")
    if args.warmup < 3:
        args.warmup = 3
    if args.study:
        run_study(args)
    elif args.oracle_rate_only:
        run_oracle_rate_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
