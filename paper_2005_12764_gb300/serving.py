"""Request loop of the serving engine (lbm_engine_* in include/lbm.h).

Requests (independent droplet or sheared-droplet design runs of different box
sizes) arrive on a seeded Poisson schedule. The loop submits each request when its
arrival time has passed, runs engine ticks (admission by device memory, batched
steps of every resident lattice, retirement of finished ones), and records each
request's latency from arrival to the end of the tick that retired it. All stepping
happens in the CUDA library; this module only schedules and measures.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs, lbm


def request_lattice(req, storage="fp16"):
    """Parameters and initial fields of one request: a droplet of radius L/4 centred
    in a periodic L^3 box (rho_r = 1 inside, rho_b = 1 outside); sheared requests
    add the Kolmogorov force 1e-5 sin(2 pi y / L)."""
    L = int(req["L"])
    c = L / 2.0
    rr, rb = inputs.paint_droplets((L, L, L), [(c, c, c, req["R"])])
    params = lbm.make_params(L, L, L, tau_r=1.0, sigma=req["sigma"], beta=0.7, A_nc=0.0,
                             kolmogorov_amp=1e-5 if req["sheared"] else 0.0, storage=storage)
    return params, rr, rb


def percentile(values, q):
    """q-th percentile (0..100) by linear interpolation between order statistics."""
    v = np.sort(np.asarray(values, dtype=np.float64))
    if v.size == 0:
        return float("nan")
    pos = (v.size - 1) * q / 100.0
    lo = int(np.floor(pos))
    hi = min(lo + 1, v.size - 1)
    return float(v[lo] + (v[hi] - v[lo]) * (pos - lo))


def serve(engine: "lbm.Engine", requests, storage="fp16", clock=time.perf_counter,
          keep_results=False):
    """Runs the request stream through the engine in real time.

    requests: dicts with arrival_s, L, R, sigma, steps, sheared (inputs.serving_requests).
    Returns a report with per-request latencies (s), p50/p99 (ms), aggregate GLUPS
    over the whole run, and the engine counters; with keep_results the fields of
    every request are returned too (keyed by the request's id).
    """
    order = sorted(range(len(requests)), key=lambda k: requests[k]["arrival_s"])
    prepared = {k: request_lattice(requests[k], storage) for k in order}
    n = len(order)
    nxt = 0
    outstanding = {}            # ticket -> request index
    latency = {}
    results = {}
    t0 = clock()
    while len(latency) < n:
        now = clock() - t0
        while nxt < n and requests[order[nxt]]["arrival_s"] <= now:
            k = order[nxt]
            params, rr, rb = prepared[k]
            t = engine.submit(params, rr, rb, requests[k]["steps"])
            outstanding[t] = k
            nxt += 1
        resident, queued, retired, _ = engine.tick()
        if retired:
            t_done = clock() - t0
            for t in [t for t in outstanding if engine.state(t) in ("finished", "failed")]:
                k = outstanding.pop(t)
                if engine.state(t) == "failed":
                    raise RuntimeError(f"request {k} failed in the engine")
                res = engine.result(t)
                latency[k] = t_done - requests[k]["arrival_s"]
                if keep_results:
                    results[requests[k]["id"]] = res
        if resident == 0 and queued == 0 and nxt < n:
            wait = requests[order[nxt]]["arrival_s"] - (clock() - t0)
            if wait > 0:
                time.sleep(wait)
    wall = clock() - t0
    first = min(r["arrival_s"] for r in requests)
    lups = sum(int(r["L"]) ** 3 * int(r["steps"]) for r in requests)
    lat = [latency[k] for k in range(n)]
    report = {
        "requests": n,
        "p50_ms": percentile(lat, 50) * 1e3,
        "p99_ms": percentile(lat, 99) * 1e3,
        "mean_ms": float(np.mean(lat)) * 1e3,
        "wall_s": wall,
        "glups": lups / (wall - first) / 1e9,
        "lattice_updates": lups,
        "latency_s": lat,
        "engine": engine.stats(),
    }
    if keep_results:
        report["results"] = results
    return report
