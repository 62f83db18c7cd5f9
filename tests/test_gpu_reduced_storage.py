"""GPU checks of the reduced (Q + 5) FP32 storage form.

The form stores each node's 19 total populations and its five recolouring
coefficients (kappa_r, kappa_b, m) instead of 2 x 19 species populations; the pull
splits every streamed total with the coefficients of its source node. It is exact,
so it is held to the FP32 bars of the full form against the FP64 oracle (after 100
steps max|d rho| <= 1e-5 per species, max|d u| <= 1e-6) on walled, sliding, ragged,
near-contact, unequal-viscosity, pinned and chain-mode lattices, and, beside the full
FP32 form, on the full-size channel workload.
"""
import numpy as np
import pytest

import oracle
from paper_2005_12764_gb300 import inputs

pytestmark = pytest.mark.gpu

RHO_TOL, U_TOL = 1e-5, 1e-6
Q5 = "fp32_q5"


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12764_gb300 import build_lib, lbm as L
    build_lib.build()
    L.load()
    return L


def run_pair(lbm, shape, fields, steps, pins=None, **kw):
    nz, ny, nx = shape
    o = oracle.Lattice(oracle.make_params(nx, ny, nz, **kw))
    o.set_fields(*fields)
    if pins is not None:
        o.set_pins(pins)
    o.step(steps)
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, storage=Q5, **kw))
    g.set_fields(*fields)
    if pins is not None:
        g.set_pin_mask(pins)
    g.step(steps)
    fo, fg = o.get_fields(), g.get_fields()
    o.close()
    g.close()
    return fo, fg


def assert_parity(fo, fg, rho_tol=RHO_TOL, u_tol=U_TOL):
    e = {k: float(np.abs(fo[k] - fg[k]).max()) for k in ("rho_r", "rho_b", "u", "phi")}
    assert e["rho_r"] <= rho_tol and e["rho_b"] <= rho_tol, e
    assert e["u"] <= u_tol, e


def test_static_droplet(lbm):
    w = inputs.static_droplet(L=32, R=8.0)
    assert_parity(*run_pair(lbm, w.shape, (w.rho_r, w.rho_b), 100, **w.params))


def test_walls_forces_near_contact_ragged_tiles(lbm):
    shape = (13, 29, 45)
    drops = [(12.0, 10.0, 6.0, 5.0), (24.5, 18.0, 6.5, 5.5), (38.0, 9.0, 6.0, 4.5)]
    rr, rb = inputs.paint_droplets(shape, drops, periodic=(True, False, False))
    kw = dict(wall_y=1, wall_z=1, sigma=0.02, beta=0.7, A_nc=0.02, h_min=3.0, g=(1e-5, 0, 0))
    assert_parity(*run_pair(lbm, shape, (rr, rb), 100, **kw))


def test_sliding_walls_sheared_droplets(lbm):
    shape = (14, 30, 50)
    drops = [(14.0, 12.0, 7.0, 5.5), (27.0, 17.0, 6.5, 5.0)]
    rr, rb = inputs.paint_droplets(shape, drops, periodic=(True, False, False))
    kw = dict(wall_y=1, wall_z=1, wall_u=0.02, sigma=0.02, beta=0.7, A_nc=0.02, h_min=3.0)
    assert_parity(*run_pair(lbm, shape, (rr, rb), 100, **kw))


def test_unequal_viscosities_kolmogorov_initial_velocity(lbm):
    shape = (24, 20, 36)
    rr, rb, u = inputs.random_state(shape, seed=21, u_amp=0.01)
    kw = dict(tau_r=0.8, tau_b=1.3, sigma=0.015, beta=0.7, kolmogorov_amp=1e-4)
    assert_parity(*run_pair(lbm, shape, (rr, rb, u), 100, **kw))


@pytest.mark.parametrize("shape", [(1, 1, 4), (3, 1, 5), (1, 6, 1), (7, 3, 5), (2, 2, 2)])
def test_degenerate_and_tiny_boxes(lbm, shape):
    rr, rb, u = inputs.random_state(shape, seed=sum(shape), u_amp=0.01)
    assert_parity(*run_pair(lbm, shape, (rr, rb, u), 20, sigma=0.02, beta=0.7))


def test_pinning_sites(lbm):
    shape = (24, 24, 24)
    rr, rb = inputs.paint_droplets(shape, [(12.0, 12.0, 12.0, 6.0)])
    rng = np.random.default_rng(17)
    pins = np.zeros(shape, np.uint8)
    for _ in range(12):
        d = rng.normal(size=3)
        pt = np.array([12.0, 12.0, 12.0]) + d / np.linalg.norm(d) * rng.uniform(4, 10)
        x, y, z = np.round(pt).astype(int) % 24
        pins[z, y, x] = 1
    kw = dict(sigma=0.01, beta=0.7, A_nc=0.01, h_min=3.0)
    assert_parity(*run_pair(lbm, shape, (rr, rb), 60, pins=pins, **kw))


def test_chain_mode_walls_ragged_near_contact(lbm):
    # 150 x 60 x 64: the step kernel runs in chain mode (runs of planes crossing
    # from one tile to the next)
    shape = (64, 60, 150)
    drops = [(20.0, 12.0, 30.0, 6.0), (33.5, 24.0, 31.0, 6.5), (50.0, 30.0, 50.0, 7.0),
             (110.0, 40.0, 20.0, 8.0), (130.0, 20.0, 55.0, 6.0)]
    rr, rb = inputs.paint_droplets(shape, drops, periodic=(True, False, False))
    kw = dict(wall_y=1, wall_z=1, sigma=0.02, beta=0.7, A_nc=0.02, h_min=3.0, g=(1e-5, 0, 0))
    assert_parity(*run_pair(lbm, shape, (rr, rb), 30, **kw))


def test_full_channel_both_forms_match_the_oracle(lbm):
    # 256 x 128 x 64 channel, 100 steps: the reduced and the full FP32 form both within
    # the FP32 bars of the FP64 oracle (they differ from each other only in rounding:
    # one multiply-add per pulled population), and species masses conserved
    w = inputs.channel_droplets()
    nz, ny, nx = w.shape
    o = oracle.Lattice(oracle.make_params(nx, ny, nz, **w.params))
    o.set_fields(w.rho_r, w.rho_b)
    o.step(100)
    fo = o.get_fields()
    o.close()
    m0 = (float(w.rho_r.sum()), float(w.rho_b.sum()))
    for st in ("fp32", Q5):
        g = lbm.Lattice(lbm.make_params(nx, ny, nz, storage=st, **w.params))
        g.set_fields(w.rho_r, w.rho_b)
        g.step(100)
        fg = g.get_fields()
        t = g.observables()
        g.close()
        assert_parity(fo, fg)
        assert abs(t[0] - m0[0]) / m0[0] < 1e-6 and abs(t[1] - m0[1]) / m0[1] < 1e-6, st


def test_pops_are_recoloured_and_survive_a_round_trip(lbm):
    # get_pops rebuilds both species; set_pops of those values stores the same
    # coefficients (the split is of the recoloured form), so the two lattices then
    # step alike; a state of the full FP32 form moved into the reduced form steps
    # like the full form
    w = inputs.channel_droplets(nx=64, ny=40, nz=24, n_grid=(2, 2, 1), r_range=(4, 6), seed=5)
    P5 = lbm.make_params(64, 40, 24, storage=Q5, **w.params)
    P32 = lbm.make_params(64, 40, 24, storage="fp32", **w.params)
    a = lbm.Lattice(P5)
    a.set_fields(w.rho_r, w.rho_b)
    a.step(10)
    fr, fb, lag = a.get_pops()
    b = lbm.Lattice(P5)
    b.set_fields(w.rho_r, w.rho_b)
    b.set_pops(fr, fb, lag)
    fr2, fb2, lag2 = b.get_pops()
    assert np.array_equal(lag, lag2)
    assert np.abs(fr2 - fr).max() <= 1e-7 and np.abs(fb2 - fb).max() <= 1e-7
    a.step(20)
    b.step(20)
    fa, fbb = a.get_fields(), b.get_fields()
    for k in ("rho_r", "rho_b", "u"):
        assert np.abs(fa[k] - fbb[k]).max() <= 1e-6, k
    c = lbm.Lattice(P32)
    c.set_fields(w.rho_r, w.rho_b)
    c.step(10)
    cr, cb, clag = c.get_pops()
    d = lbm.Lattice(P5)
    d.set_fields(w.rho_r, w.rho_b)
    d.set_pops(cr, cb, clag)
    c.step(20)
    d.step(20)
    fc, fd = c.get_fields(), d.get_fields()
    for k in ("rho_r", "rho_b", "u"):
        assert np.abs(fc[k] - fd[k]).max() <= 1e-6, k
    for g in (a, b, c, d):
        g.close()


def test_checkpoint_resume_is_bitwise(lbm):
    w = inputs.channel_droplets(nx=64, ny=40, nz=24, n_grid=(2, 2, 1), r_range=(4, 6), seed=5)
    P = lbm.make_params(64, 40, 24, storage=Q5, **w.params)
    a = lbm.Lattice(P)
    a.set_fields(w.rho_r, w.rho_b)
    a.step(30)
    blob = a.save_state()
    a.step(30)
    b = lbm.Lattice(P)
    b.load_state(blob)
    b.step(30)
    pa, pb = a.get_pops(), b.get_pops()
    assert all(np.array_equal(x, y) for x, y in zip(pa, pb))
    a.close()
    b.close()


def test_shan_chen_is_refused(lbm):
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(lbm.make_params(16, 16, 16, storage=Q5, model="shan_chen", G_sc=1.2))


def test_zero_steps_returns_set_fields(lbm):
    # f^eq(rho_k, u) is (rho_k / rho) f^eq(rho, u): the reduced form holds any initial
    # state exactly up to FP32 rounding
    shape = (5, 6, 7)
    rr, rb, u = inputs.random_state(shape, seed=3)
    g = lbm.Lattice(lbm.make_params(7, 6, 5, storage=Q5))
    g.set_fields(rr, rb, u)
    g.step(0)
    f = g.get_fields()
    g.close()
    assert np.abs(f["rho_r"] - rr).max() < 4e-7 and np.abs(f["rho_b"] - rb).max() < 4e-7
    assert np.abs(f["u"] - u).max() < 1e-7


def test_laplace_and_observables_match_the_oracle(lbm):
    w = inputs.static_droplet(L=32, R=8.0)
    o = oracle.Lattice(oracle.make_params(32, 32, 32, **w.params))
    o.set_fields(w.rho_r, w.rho_b)
    o.step(200)
    g = lbm.Lattice(lbm.make_params(32, 32, 32, storage=Q5, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    t0 = g.observables()
    g.step(200)
    lo, lg = o.laplace((16, 16, 16)), g.laplace((16, 16, 16))
    assert abs(lg["R_eff"] - lo["R_eff"]) < 1e-4
    assert abs(lg["dp"] - lo["dp"]) / abs(lo["dp"]) < 1e-3
    t = g.observables()
    assert abs(t[0] - t0[0]) / t0[0] < 1e-6 and abs(t[1] - t0[1]) / t0[1] < 1e-6
    assert np.abs(t[2:5]).max() / (t0[0] + t0[1]) < 1e-7
    o.close()
    g.close()


def test_window_matches_full_download_with_wrap(lbm):
    g = lbm.Lattice(lbm.make_params(16, 10, 12, sigma=0.01, storage=Q5))
    rr, rb = inputs.paint_droplets((12, 10, 16), [(8.0, 5.0, 6.0, 3.5)])
    g.set_fields(rr, rb)
    g.step(5)
    fr, fb, lag = g.get_pops()
    wr, wb, wl = g.get_window(13, 7, 9, 6, 5, 4)
    zz = (np.arange(9, 13) % 12)[:, None, None]
    yy = (np.arange(7, 12) % 10)[None, :, None]
    xx = (np.arange(13, 19) % 16)[None, None, :]
    assert np.array_equal(wr.reshape(19, 4, 5, 6), fr[:, zz, yy, xx])
    assert np.array_equal(wb.reshape(19, 4, 5, 6), fb[:, zz, yy, xx])
    assert np.array_equal(wl.reshape(4, 5, 6), lag[zz, yy, xx])
    g.close()


# ---------------------------------------------------------------- FP16 reduced form
# The 19 totals in FP16 as deviations from w_i rho0, the coefficients exact: held to
# the bars of FP16 storage (rho within 1e-3 of the oracle after 100 steps, the Laplace
# pressure jump within 2 %).
Q5H = "fp16_q5"


def run_pair_h(lbm, shape, fields, steps, pins=None, **kw):
    nz, ny, nx = shape
    o = oracle.Lattice(oracle.make_params(nx, ny, nz, **kw))
    o.set_fields(*fields)
    if pins is not None:
        o.set_pins(pins)
    o.step(steps)
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, storage=Q5H, **kw))
    g.set_fields(*fields)
    if pins is not None:
        g.set_pin_mask(pins)
    g.step(steps)
    out = o.get_fields(), g.get_fields(), o.totals(), g.observables()
    o.close()
    g.close()
    return out


@pytest.mark.parametrize("case", ["droplet", "walls_nc", "sliding_unequal_tau"])
def test_fp16_reduced_form_accuracy(lbm, case):
    if case == "droplet":
        w = inputs.static_droplet(L=32, R=8.0)
        shape, fields, kw = w.shape, (w.rho_r, w.rho_b), w.params
    elif case == "walls_nc":
        shape = (13, 29, 45)
        drops = [(12.0, 10.0, 6.0, 5.0), (24.5, 18.0, 6.5, 5.5), (38.0, 9.0, 6.0, 4.5)]
        fields = inputs.paint_droplets(shape, drops, periodic=(True, False, False))
        kw = dict(wall_y=1, wall_z=1, sigma=0.02, beta=0.7, A_nc=0.02, h_min=3.0, g=(1e-5, 0, 0))
    else:
        shape = (14, 30, 50)
        drops = [(14.0, 12.0, 7.0, 5.5), (27.0, 17.0, 6.5, 5.0)]
        fields = inputs.paint_droplets(shape, drops, periodic=(True, False, False))
        kw = dict(wall_y=1, wall_z=1, wall_u=0.02, sigma=0.02, beta=0.7, A_nc=0.02, h_min=3.0,
                  tau_r=0.8, tau_b=1.3)
    fo, fg, to, tg = run_pair_h(lbm, shape, fields, 100, **kw)
    e = {k: float(np.abs(fo[k] - fg[k]).max()) for k in ("rho_r", "rho_b", "u")}
    print(case, e)
    assert e["rho_r"] <= 1e-3 and e["rho_b"] <= 1e-3, e
    # the coefficients are exact: the species masses move only by the rounding of the
    # FP16 totals, far below the density bar
    for k in range(2):
        assert abs(tg[k] - to[k]) / to[k] < 1e-4, (k, tg[k], to[k])


def test_fp16_reduced_form_laplace_pressure_jump(lbm):
    w = inputs.static_droplet(L=32, R=8.0)
    n = 32
    o = oracle.Lattice(oracle.make_params(n, n, n, **w.params))
    o.set_fields(w.rho_r, w.rho_b)
    o.step(500)
    lo = o.laplace((16.0, 16.0, 16.0))
    g = lbm.Lattice(lbm.make_params(n, n, n, storage=Q5H, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    g.step(500)
    lg = g.laplace((16.0, 16.0, 16.0))
    g.close()
    assert abs(lg["dp"] - lo["dp"]) / lo["dp"] < 0.02, (lg, lo)
