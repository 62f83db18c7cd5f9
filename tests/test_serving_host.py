"""Host-side pieces of the serving layer (no GPU): the seeded request stream and
the latency statistics."""
import numpy as np

from paper_2005_12764_gb300 import inputs, serving


def test_percentile_matches_numpy_linear():
    rng = np.random.default_rng(3)
    v = rng.exponential(size=101)
    for q in (0, 1, 50, 99, 100):
        assert abs(serving.percentile(v, q) - np.percentile(v, q)) < 1e-12


def test_request_stream_is_seeded_poisson_with_the_stated_mix():
    a = inputs.serving_requests()
    b = inputs.serving_requests()
    assert a == b and len(a) == 256
    t = np.array([r["arrival_s"] for r in a])
    gaps = np.diff(t)
    assert (gaps >= 0).all()
    # mean inter-arrival 1/50 s within sampling error (sd / sqrt(255) ~ 1.3e-3)
    assert abs(gaps.mean() - 0.02) < 0.005
    assert {r["L"] for r in a} <= {32, 48, 64, 96, 128}
    assert all(r["R"] == r["L"] / 4 and 200 <= r["steps"] <= 2000 for r in a)
    assert all(0.005 <= r["sigma"] <= 0.03 for r in a)
    frac = np.mean([r["sheared"] for r in a])
    assert 0.35 < frac < 0.65


def test_request_lattice_is_a_centred_droplet():
    req = dict(id=0, L=32, R=8.0, sigma=0.01, steps=10, sheared=True)
    p, rr, rb = serving.request_lattice(req)
    assert (p.nx, p.ny, p.nz) == (32, 32, 32) and p.storage == 1
    assert p.kolmogorov_amp == 1e-5 and p.A_nc == 0.0
    vol = rr.sum()
    assert abs(vol - 4.0 / 3.0 * np.pi * 8 ** 3) / vol < 0.05
    assert np.allclose(rr + rb, 1.0)
