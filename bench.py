"""Benchmark of the fused colour-gradient LB step on GB300.

Default workload: the microfluidic-crystal channel, 256 x 128 x 64 D3Q19 nodes with
bounce-back walls at the y and z extremes, 40 droplets (radii 6-9, seeded), sigma =
0.02, beta = 0.7, near-contact force A = 0.01 within 3 lu, g_x = 1e-6, FP32 storage.
One step = one lattice update of every node (one launch of the fused kernel).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--storage fp32|fp16|bf16|fp32_q5]
                  [--impl ours|reference] [--model colour|shan_chen] [--no-serving]
                  [--no-models] [--no-cpu-baseline]

Prints one JSON line. ``value`` is GLUPS (10^9 lattice-node updates per second)
over all ranks; ``e2e`` times the same job through the public C-ABI with host
buffers (set fields from pinned host memory, K steps, fields back to the host);
``roofline`` relates the step kernel's algorithmic bytes (2 x 19 x 2 populations
per node, read once and written once) to the measured HBM bandwidth;
``fp16_store`` repeats the device-resident measurement with FP16 deviation
storage (and, inside it, BF16) and ``fp32_q5_store`` with the reduced FP32 form (19 totals and 5 recolouring
coefficients per node, 2 x 24 x 4 bytes per node and step); ``serving`` runs the served request stream (256 droplet / sheared-droplet
runs of edge 32-128, Poisson arrivals at 50/s, FP16 storage) through the serving
engine and reports p50/p99 latency beside aggregate GLUPS; ``shan_chen`` and
``sheared_bijel`` give the device-resident GLUPS of the Shan-Chen model on the same
channel and of the sheared-bijel channel with sliding walls; ``cpu_baseline`` times
the FP64 oracle on the host cores. ``--impl reference`` times the oracle itself on
the same workload (the method has no other reference implementation). Multi-GPU
runs are independent replicas: one channel lattice per rank, the request stream
sharded over the ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS & % HBM roofline, FP32 vs FP16-store; served-run p50/p99 latency"
WORKLOAD = "microfluidic-crystal channel 256x128x64, 40 droplets, walls y/z, NC on"
Q, C = 19, 2


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
    written once (2 x 2Q values, or 2 x (Q + 5) in the reduced FP32 form)."""
    if storage == "fp32_q5":
        return 2 * (Q + 5) * 4
    return 2 * Q * C * (4 if storage == "fp32" else 2)


def measured_traffic(storage: str):
    """DRAM bytes per launch of the step kernel from the committed ncu summary, if it
    was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and not line.startswith("#") and parts[0] == want and parts[1] == storage:
            return float(parts[2])
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms in a thread."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if s[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def bench_workload(args):
    """The timed workload: the channel, with the colour-gradient model (default) or the
    Shan-Chen model (--model shan_chen)."""
    from paper_2005_12764_gb300 import inputs
    if args.model == "shan_chen":
        return inputs.channel_shan_chen()
    return inputs.channel_droplets()


def workload_name(args):
    if args.model == "shan_chen":
        return "microfluidic-crystal channel 256x128x64, 40 droplets, walls y/z, Shan-Chen G_sc = 1.6"
    return WORKLOAD


def cpu_oracle_rate(workload, steps, warm=1):
    """Oracle lattice updates per second on this host (all cores) over `steps` steps."""
    import oracle
    nz, ny, nx = workload.shape
    lat = oracle.Lattice(oracle.make_params(nx, ny, nz, **workload.params))
    lat.set_fields(workload.rho_r, workload.rho_b)
    lat.step(warm)
    t0 = time.perf_counter()
    lat.step(steps)
    dt = time.perf_counter() - t0
    lat.close()
    return nx * ny * nz * steps / dt, dt


def run_reference(args):
    """The FP64 oracle timed on the host cores, on the same workload and metric."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = bench_workload(args)
    N = w.rho_r.size
    import oracle
    nz, ny, nx = w.shape
    lat = oracle.Lattice(oracle.make_params(nx, ny, nz, **w.params))
    lat.set_fields(w.rho_r, w.rho_b)
    lat.step(args.warmup)
    t0 = time.perf_counter()
    lat.step(args.steps)
    dt = time.perf_counter() - t0
    glups = N * args.steps / dt / 1e9
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": glups, "unit": "GLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args), "nodes": N, "storage": "f64 (oracle)"},
            "cpu_baseline": {"value": glups, "unit": "GLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full steps of the {nx}x{ny}x{nz} channel"},
            "e2e": {"value": glups, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def device_resident_glups(lbm, w, storage, steps, warmup, stream, local):
    """GLUPS of `steps` steps queued back to back (CUDA events on the library's
    stream) and the mean step-kernel time (ms) from the library's own events."""
    import torch
    nz, ny, nx = w.shape
    lat = lbm.Lattice(lbm.make_params(nx, ny, nz, storage=storage, stream=stream.cuda_stream,
                                      **w.params))
    lat.set_fields(torch.from_numpy(w.rho_r).to(f"cuda:{local}"),
                   torch.from_numpy(w.rho_b).to(f"cuda:{local}"))
    lat.step(warmup)
    lat.sync()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    lat.step(steps)
    b.record(stream)
    stream.synchronize()
    ms = a.elapsed_time(b)
    kt = max(5, min(steps, 50))
    _, step_ms, _ = lat.step_timed(kt)
    lat.close()
    return nx * ny * nz * steps / (ms * 1e-3) / 1e9, ms / steps, step_ms / kt


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


def other_workloads(lbm, stream, local, steps=200):
    """Device-resident GLUPS of two more workloads of the same step: the Shan-Chen
    model on the channel geometry, and the sheared-bijel channel (1024 x 128 x 128,
    sliding walls, near contact on) after 300 steps of coarsening from the quench."""
    import torch
    from paper_2005_12764_gb300 import inputs
    out = {}

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
    ms = timed(lat, steps)
    _, k_ms, _ = lat.step_timed(20)
    lat.close()
    alg = bytes_per_node("fp32") * nx * ny * nz
    out["shan_chen"] = {"workload": "channel 256x128x64, 40 droplets, walls y/z, G_sc = 1.6, FP32",
                        "value": nx * ny * nz / (ms * 1e-3) / 1e9, "unit": "GLUPS",
                        "ms_per_step": ms, "kernel_ms": k_ms / 20,
                        "roofline_frac": alg / (k_ms / 20 * 1e-3) / 1e9 / peaks()[0],
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

    from paper_2005_12764_gb300 import build_lib, inputs, lbm, replicas

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build_lib.build()
    w = bench_workload(args)
    nz, ny, nx = w.shape
    N = nx * ny * nz
    stream = torch.cuda.Stream()
    P = lbm.make_params(nx, ny, nz, storage=args.storage, stream=stream.cuda_stream, **w.params)
    lat = lbm.Lattice(P)
    dev_rr = torch.from_numpy(w.rho_r).to(f"cuda:{local}")
    dev_rb = torch.from_numpy(w.rho_b).to(f"cuda:{local}")
    torch.cuda.synchronize()
    lat.set_fields(dev_rr, dev_rb)
    lat.step(args.warmup)
    lat.sync()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timing: K steps queued back to back, CUDA events on the
    # stream the kernels run on
    barrier()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        lat.step(args.steps)
        t_end.record(stream)
        stream.synchronize()
    barrier()
    total_ms = replicas.max_over_ranks(t_start.elapsed_time(t_end), dist if world > 1 else None,
                                       f"cuda:{local}")
    ms_per_step = total_ms / args.steps
    glups = world * N * args.steps / (total_ms * 1e-3) / 1e9
    # per-kernel durations (events around each launch, inside the library)
    kt = max(5, min(args.steps, 50))
    nc_ms, step_ms, _ = lat.step_timed(kt)
    kern_ms = [step_ms / kt]
    nc_avg_ms = nc_ms / kt
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

    # ---- roofline of the step kernel
    alg_bytes = bytes_per_node(args.storage) * N
    k_avg = statistics.mean(kern_ms) * 1e-3
    achieved = alg_bytes / k_avg / 1e9
    peak, peak_kind = peaks()
    traffic = measured_traffic(args.storage)

    obs = lat.observables()
    finite = bool(np.isfinite(obs[:5]).all())
    launches = args.steps * lat.launches_per_step
    lat.close()
    # the same workload with FP16 deviation storage (device-resident, as `value`)
    fp16 = q5 = None
    if args.storage == "fp32":
        g16, ms16, k16 = device_resident_glups(lbm, w, "fp16", args.steps, args.warmup, stream, local)
        g16 = replicas.sum_over_ranks(g16, dist if world > 1 else None, f"cuda:{local}")
        alg16 = 2 * Q * C * 2 * N
        fp16 = {"value": g16, "unit": "GLUPS", "ms_per_step": ms16, "kernel_ms": k16,
                "roofline_frac": alg16 / (k16 * 1e-3) / 1e9 / peaks()[0],
                "algorithmic_bytes_per_launch": alg16}
        # BF16 deviation storage beside it (same bytes, 8-bit mantissa)
        gb, msb, kb = device_resident_glups(lbm, w, "bf16", args.steps, args.warmup, stream, local)
        gb = replicas.sum_over_ranks(gb, dist if world > 1 else None, f"cuda:{local}")
        fp16["bf16"] = {"value": gb, "unit": "GLUPS", "ms_per_step": msb, "kernel_ms": kb}
    if args.storage == "fp32" and args.model == "colour":
        # and with the reduced FP32 form (Q + 5 values per node; colour-gradient states
        # only), against its own byte model of 192 bytes per node and step
        g5, ms5, k5 = device_resident_glups(lbm, w, "fp32_q5", args.steps, args.warmup, stream,
                                            local)
        g5 = replicas.sum_over_ranks(g5, dist if world > 1 else None, f"cuda:{local}")
        alg5 = bytes_per_node("fp32_q5") * N
        q5 = {"value": g5, "unit": "GLUPS", "ms_per_step": ms5, "kernel_ms": k5,
              "roofline_frac": alg5 / (k5 * 1e-3) / 1e9 / peaks()[0],
              "algorithmic_bytes_per_launch": alg5, "traffic": measured_traffic("fp32_q5")}
    others = None
    if not args.no_models:
        others = other_workloads(lbm, stream, local)
    serving_rep = None
    if not args.no_serving:
        serving_rep = serving_run(lbm, rank, world, dist if world > 1 else None, local)
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            rate, dt = cpu_oracle_rate(w, args.cpu_steps)
            cpu = {"value": rate / 1e9, "unit": "GLUPS", "cores": os.cpu_count(),
                   "kind": "oracle",
                   "sample": f"{args.cpu_steps} full FP64 steps of the {nx}x{ny}x{nz} channel "
                             f"({dt:.1f} s)"}
        line = {
            "metric": METRIC, "value": glups, "unit": "GLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args), "nodes": N, "storage": args.storage,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (%.0f MB of populations per copy)"
                             % (bytes_per_node(args.storage) * N / 2 / 1e6)},
            "e2e": {"value": e2e, "unit": "GLUPS",
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "job": "set_fields(host) + K steps + get_fields(host)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} HBM copy bandwidth",
                         "kernel": "step_kernel (fused stream/collide/perturb/recolour)",
                         "kernel_ms": statistics.mean(kern_ms),
                         "near_contact_pass_ms": nc_avg_ms,
                         "ghost_fill": "written by the near-contact pass (no launch of its own)",
                         "algorithmic_bytes_per_launch": alg_bytes},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "finite": finite,
        }
        if fp16:
            line["fp16_store"] = fp16
        if q5:
            line["fp32_q5_store"] = q5
        if others:
            line.update(others)
        if serving_rep:
            line["serving"] = serving_rep
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16", "bf16", "fp32_q5"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--model", default="colour", choices=["colour", "shan_chen"],
                    help="model of the timed workload (default: the colour-gradient channel)")
    ap.add_argument("--no-models", action="store_true",
                    help="skip the Shan-Chen and sheared-bijel lines")
    args = ap.parse_args()
    if args.storage == "fp32_q5" and args.model == "shan_chen":
        ap.error("the reduced storage form holds colour-gradient states only")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
