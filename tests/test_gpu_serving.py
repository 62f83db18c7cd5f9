"""Serving engine on the GPU (lbm_engine_*): batched, graph-captured stepping of
many resident lattices, admission by device memory, continuous batching.

The bar: a request's result is the same alone and in any mix -- here bitwise,
since every node is computed by the same arithmetic whatever the batch -- and the
same as a plain context stepped by lbm_step.
"""
import numpy as np
import pytest

from paper_2005_12764_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12764_gb300 import build_lib, lbm as L
    build_lib.build()
    L.load()
    return L


REQS = [dict(id=0, L=32, R=8.0, sigma=0.02, steps=37, sheared=False),
        dict(id=1, L=48, R=12.0, sigma=0.01, steps=64, sheared=True),
        dict(id=2, L=32, R=8.0, sigma=0.005, steps=90, sheared=True),
        dict(id=3, L=40, R=10.0, sigma=0.03, steps=51, sheared=False)]


def _run_alone(lbm, serving, req, storage):
    e = lbm.Engine(budget_bytes=8 << 30, max_slots=1, chunk_steps=16, autotune=False)
    p, rr, rb = serving.request_lattice(req, storage)
    t = e.submit(p, rr, rb, req["steps"])
    while e.state(t) != "finished":
        e.tick()
    out = e.result(t)
    e.close()
    return out


@pytest.mark.parametrize("storage", ["fp16", "fp32", "fp32_q5", "fp16_q5"])
def test_result_is_the_same_alone_in_the_mix_and_by_lbm_step(lbm, storage):
    from paper_2005_12764_gb300 import serving
    alone = {r["id"]: _run_alone(lbm, serving, r, storage) for r in REQS}
    # the mix: two requests first, the others arrive while those are resident
    e = lbm.Engine(budget_bytes=8 << 30, max_slots=8, chunk_steps=12, autotune=True)
    tickets = {}
    for r in REQS[:2]:
        p, rr, rb = serving.request_lattice(r, storage)
        tickets[e.submit(p, rr, rb, r["steps"])] = r["id"]
    e.tick()
    e.tick()
    for r in REQS[2:]:
        p, rr, rb = serving.request_lattice(r, storage)
        tickets[e.submit(p, rr, rb, r["steps"])] = r["id"]
    mixed = {}
    for _ in range(200):
        e.tick()
        for t, k in tickets.items():
            if k not in mixed and e.state(t) == "finished":
                mixed[k] = e.result(t)
        if len(mixed) == len(REQS):
            break
    e.close()
    assert len(mixed) == len(REQS)
    for r in REQS:
        a, m = alone[r["id"]], mixed[r["id"]]
        assert a["info"][0] == m["info"][0] == r["steps"]
        for key in ("rho_r", "rho_b", "u", "phi"):
            assert np.array_equal(a[key], m[key]), (r["id"], key)
        # and the same as a plain context stepped by lbm_step
        p, rr, rb = serving.request_lattice(r, storage)
        g = lbm.Lattice(p)
        g.set_fields(rr, rb)
        g.step(r["steps"])
        f = g.get_fields()
        g.close()
        for key in ("rho_r", "rho_b", "u", "phi"):
            assert np.array_equal(f[key], m[key]), (r["id"], key, "lbm_step")


def test_admission_by_device_memory(lbm):
    from paper_2005_12764_gb300 import serving
    reqs = [dict(id=k, L=48, R=12.0, sigma=0.01, steps=20, sheared=bool(k % 2)) for k in range(6)]
    p, _, _ = serving.request_lattice(reqs[0])
    one = lbm.footprint_bytes(p) + 7 * 48 ** 3 * 8        # a request's device memory
    budget = int(2.5 * one)                                  # room for two at a time
    e = lbm.Engine(budget_bytes=budget, max_slots=16, chunk_steps=8, autotune=False)
    tickets = []
    for r in reqs:
        p, rr, rb = serving.request_lattice(r)
        tickets.append(e.submit(p, rr, rb, r["steps"]))
    seen_queue = 0
    for _ in range(100):
        res, q, _, _ = e.tick()
        assert res <= 2
        seen_queue = max(seen_queue, q)
        if all(e.state(t) == "finished" for t in tickets):
            break
    st = e.stats()
    assert all(e.state(t) == "finished" for t in tickets)
    assert seen_queue >= 3 and st["peak_bytes"] <= budget
    # a request larger than the whole budget is refused at submission
    big = lbm.make_params(256, 256, 256, storage="fp16")
    with pytest.raises(lbm.LbmError):
        e.submit(big, np.ones(256 ** 3), np.zeros(256 ** 3), 10)
    e.close()


def test_serving_loop_reports_latency_and_throughput(lbm):
    from paper_2005_12764_gb300 import serving
    reqs = inputs.serving_requests(n=24, seed=7, rate_hz=400.0, edges=(32, 48, 64),
                                   steps_range=(40, 160))
    e = lbm.Engine(budget_bytes=16 << 30, max_slots=32, chunk_steps=20)
    rep = serving.serve(e, reqs, storage="fp16")
    e.close()
    assert rep["requests"] == 24 and len(rep["latency_s"]) == 24
    assert 0 < rep["p50_ms"] <= rep["p99_ms"]
    assert rep["glups"] > 0
    print("serving report:", {k: v for k, v in rep.items() if k != "latency_s"})


def test_shortest_job_first_admission(lbm):
    from paper_2005_12764_gb300 import serving
    big = dict(id=0, L=48, R=12.0, sigma=0.01, steps=60, sheared=False)
    small = [dict(id=k, L=32, R=8.0, sigma=0.01, steps=10 + k, sheared=False) for k in (1, 2, 3)]
    order = []
    for policy in ("fcfs", "sjf"):
        e = lbm.Engine(budget_bytes=8 << 30, max_slots=1, chunk_steps=8, autotune=False, policy=policy)
        tickets = {}
        for r in [big] + small:          # the big request arrives first
            p, rr, rb = serving.request_lattice(r)
            tickets[e.submit(p, rr, rb, r["steps"])] = r["id"]
        done = []
        for _ in range(100):
            e.tick()
            for t, k in tickets.items():
                if k not in done and e.state(t) == "finished":
                    done.append(k)
            if len(done) == 4:
                break
        e.close()
        order.append(done)
    assert order[0] == [0, 1, 2, 3]          # first come, first served
    assert order[1] == [1, 2, 3, 0]          # shortest (fewest node-steps) first


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_shan_chen_requests_in_a_mix_are_bitwise_lbm_step(lbm, storage):
    # Shan-Chen and colour-gradient requests resident together (two batched launches
    # per step): each result equals the same lattice stepped by plain lbm_step
    from paper_2005_12764_gb300 import serving
    reqs = [dict(id=0, L=32, R=8.0, sigma=0.02, steps=30, sheared=False),
            dict(id=1, L=48, R=12.0, sigma=0.01, steps=40, sheared=True)]
    L = 40
    rr, rb = inputs.paint_droplets((L, L, L), [(20.0, 20.0, 20.0, 10.0)])
    rr, rb = 0.96 * rr + 0.02, 0.96 * rb + 0.02
    psc = lbm.make_params(L, L, L, model="shan_chen", G_sc=1.6, storage=storage,
                          kolmogorov_amp=1e-5)
    e = lbm.Engine(budget_bytes=8 << 30, max_slots=8, chunk_steps=10, autotune=False)
    tickets = {}
    for r in reqs:
        p, a, b = serving.request_lattice(r, storage)
        tickets[e.submit(p, a, b, r["steps"])] = ("cg", r, p, a, b)
    tickets[e.submit(psc, rr, rb, 35)] = ("sc", None, psc, rr, rb)
    done = {}
    for _ in range(200):
        e.tick()
        for t in tickets:
            if t not in done and e.state(t) == "finished":
                done[t] = e.result(t)
        if len(done) == len(tickets):
            break
    e.close()
    assert len(done) == len(tickets)
    for t, (kind, r, p, a, b) in tickets.items():
        g = lbm.Lattice(p)
        g.set_fields(a, b)
        g.step(r["steps"] if r else 35)
        f = g.get_fields()
        g.close()
        for k in ("rho_r", "rho_b", "u", "phi"):
            assert np.array_equal(f[k], done[t][k]), (kind, k)


def test_cancel_queued_and_resident_requests(lbm):
    # failures handled on the host: a request that can never fit, one withdrawn while
    # queued, one withdrawn while resident; the others finish bitwise as lbm_step
    from paper_2005_12764_gb300 import serving
    reqs = [dict(id=k, L=L, R=L / 4, sigma=0.02, steps=30, sheared=bool(k % 2))
            for k, L in enumerate((32, 40, 32, 48))]
    e = lbm.Engine(budget_bytes=200 << 20, max_slots=2, chunk_steps=10, autotune=False)
    big = lbm.make_params(128, 128, 128, storage="fp16")    # ~440 MB: never fits
    with pytest.raises(lbm.LbmError):
        e.submit(big, np.ones(128 ** 3), np.zeros(128 ** 3), 5)
    tk = []
    for r in reqs:
        p, a, b = serving.request_lattice(r, "fp32")
        tk.append(e.submit(p, a, b, r["steps"]))
    e.tick()                                  # requests 0, 1 resident; 2, 3 queued
    assert [e.state(t) for t in tk] == ["resident", "resident", "queued", "queued"]
    e.cancel(tk[2])                           # queued
    e.cancel(tk[1])                           # resident, mid-run
    assert e.state(tk[1]) == e.state(tk[2]) == "cancelled"
    with pytest.raises(lbm.LbmError):
        e.cancel(tk[1])
    for _ in range(50):
        e.tick()
        if all(e.state(t) in ("finished", "cancelled") for t in tk):
            break
    for k in (0, 3):
        assert e.state(tk[k]) == "finished"
        got = e.result(tk[k])
        p, a, b = serving.request_lattice(reqs[k], "fp32")
        g = lbm.Lattice(p)
        g.set_fields(a, b)
        g.step(reqs[k]["steps"])
        f = g.get_fields()
        g.close()
        for key in ("rho_r", "rho_b", "u", "phi"):
            assert np.array_equal(got[key], f[key]), (k, key)
    with pytest.raises(lbm.LbmError):
        e.result(tk[2])
    e.close()


@pytest.mark.parametrize("with_batched", [True, False])
def test_near_contact_requests_are_served_bitwise_lbm_step(lbm, with_batched):
    # near-contact requests (two droplets close enough for the film force) are batched
    # like the others: per group (storage, relaxation class, model, halo class of the
    # film rays) one near-contact launch over all its lattices precedes the batched step
    # kernel. Each result equals the same lattice stepped by plain lbm_step, beside
    # batched lattices without the force or alone; several lattices of different sizes
    # share one near-contact launch (one of them large enough for tensor-copied cubes).
    from paper_2005_12764_gb300 import serving
    nc = []
    cases = ((40, 2.0, "fp32", 3.0), (48, 3.0, "fp32_q5", 3.0), (64, 2.5, "fp32", 3.0),
             (36, 2.0, "fp32", 3.0), (44, 2.0, "fp16_q5", 3.0), (40, 2.0, "fp32", 2.0))
    for k, (L, gap, st, hmin) in enumerate(cases):
        c, R = L / 2.0, L / 6.0
        drops = [(c - R - gap / 2, c, c, R), (c + R + gap / 2, c, c, R)]
        a, b = inputs.paint_droplets((L, L, L), drops)
        p = lbm.make_params(L, L, L, sigma=0.02, beta=0.7, A_nc=0.02, h_min=hmin,
                            storage=st, kolmogorov_amp=1e-4 if k % 2 else 0.0)
        nc.append((p, a, b, 25 + 10 * (k % 3)))
    e = lbm.Engine(budget_bytes=8 << 30, max_slots=8, chunk_steps=10, autotune=False)
    tickets = {}
    for p, a, b, steps in nc:
        tickets[e.submit(p, a, b, steps)] = (p, a, b, steps)
    if with_batched:
        for r in REQS[:2]:
            p, a, b = serving.request_lattice(r, "fp32")
            tickets[e.submit(p, a, b, r["steps"])] = (p, a, b, r["steps"])
    done = {}
    for _ in range(200):
        e.tick()
        for t in tickets:
            if t not in done and e.state(t) == "finished":
                done[t] = e.result(t)
        if len(done) == len(tickets):
            break
    e.close()
    assert len(done) == len(tickets)
    for t, (p, a, b, steps) in tickets.items():
        assert done[t]["info"][0] == steps
        g = lbm.Lattice(p)
        g.set_fields(a, b)
        g.step(steps)
        f = g.get_fields()
        g.close()
        for k in ("rho_r", "rho_b", "u", "phi"):
            assert np.array_equal(f[k], done[t][k]), (t, k)
