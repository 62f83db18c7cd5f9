"""GPU parity: the CUDA library (FP32 arithmetic) against the FP64 oracle.

Bars (fixed by the method's accuracy target): after 100 steps max|d rho| <= 1e-5
for each species density and max|d u| <= 1e-6 for the physical velocity; FP16
(and BF16) deviation storage: rho within 1e-3, FP16 Laplace pressure jump within
2 %. Inputs are the seeded synthetic workloads.
"""
import math

import numpy as np
import pytest

import branch_cases
import oracle
from paper_2005_12764_gb300 import inputs

pytestmark = pytest.mark.gpu

RHO_TOL, U_TOL = 1e-5, 1e-6


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12764_gb300 import build_lib, lbm as L
    build_lib.build()
    L.load()
    return L


def run_pair(lbm, shape, fields, steps, storage="fp32", pins=None, **kw):
    nz, ny, nx = shape
    o = oracle.Lattice(oracle.make_params(nx, ny, nz, **kw))
    o.set_fields(*fields)
    if pins is not None:
        o.set_pins(pins)
    o.step(steps)
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, storage=storage, **kw))
    g.set_fields(*fields)
    if pins is not None:
        g.set_pin_mask(pins)
    g.step(steps)
    return o.get_fields(), g.get_fields(), o, g


def errs(fo, fg):
    return {k: float(np.abs(fo[k] - fg[k]).max()) for k in ("rho_r", "rho_b", "u", "phi")}


def assert_parity(fo, fg, rho_tol=RHO_TOL, u_tol=U_TOL):
    e = errs(fo, fg)
    assert e["rho_r"] <= rho_tol and e["rho_b"] <= rho_tol, e
    assert e["u"] <= u_tol, e


def test_static_droplet_100_steps(lbm):
    w = inputs.static_droplet(L=32, R=8.0)
    fo, fg, _, _ = run_pair(lbm, w.shape, (w.rho_r, w.rho_b), 100, **w.params)
    assert_parity(fo, fg)


def test_walls_forces_near_contact_ragged_tiles(lbm):
    # x, y not multiples of the 32 x 8 tile; walls in y and z; body force; near contact
    shape = (13, 29, 45)
    drops = [(12.0, 10.0, 6.0, 5.0), (24.5, 18.0, 6.5, 5.5), (38.0, 9.0, 6.0, 4.5)]
    rr, rb = inputs.paint_droplets(shape, drops, periodic=(True, False, False))
    kw = dict(wall_y=1, wall_z=1, sigma=0.02, beta=0.7, A_nc=0.02, h_min=3.0, g=(1e-5, 0, 0))
    fo, fg, _, _ = run_pair(lbm, shape, (rr, rb), 100, **kw)
    assert_parity(fo, fg)


def test_channel_workload_shape_small(lbm):
    w = inputs.channel_droplets(nx=64, ny=40, nz=24, n_grid=(2, 2, 1), r_range=(4, 6), seed=5)
    fo, fg, _, _ = run_pair(lbm, w.shape, (w.rho_r, w.rho_b), 100, **w.params)
    assert_parity(fo, fg)


def test_unequal_viscosities_and_kolmogorov(lbm):
    shape = (24, 20, 36)
    rr, rb, u = inputs.random_state(shape, seed=21, u_amp=0.01)
    kw = dict(tau_r=0.8, tau_b=1.3, sigma=0.015, beta=0.7, kolmogorov_amp=1e-4)
    fo, fg, _, _ = run_pair(lbm, shape, (rr, rb, u), 100, **kw)
    assert_parity(fo, fg)


@pytest.mark.parametrize("shape", [(1, 1, 4), (3, 1, 5), (1, 6, 1), (7, 3, 5), (2, 2, 2)])
def test_degenerate_and_tiny_boxes(lbm, shape):
    rr, rb, u = inputs.random_state(shape, seed=sum(shape), u_amp=0.01)
    kw = dict(sigma=0.02, beta=0.7)
    fo, fg, _, _ = run_pair(lbm, shape, (rr, rb, u), 20, **kw)
    assert_parity(fo, fg)


def test_pinning_sites(lbm):
    # A droplet with pinning sites scattered around its interface (distances 4-10
    # from the centre). A stable configuration: the symmetric noise quench of the
    # gel workload is a physical instability, where FP32 and FP64 runs separate
    # exponentially, so it is checked one step at a time instead (below).
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
    fo, fg, _, _ = run_pair(lbm, shape, (rr, rb), 60, pins=pins, **kw)
    assert_parity(fo, fg)


def test_sliding_walls_sheared_droplets(lbm):
    # two droplets between walls sliding with +-U along x (z walls at rest), near
    # contact on, ragged tiles
    shape = (14, 30, 50)
    drops = [(14.0, 12.0, 7.0, 5.5), (27.0, 17.0, 6.5, 5.0)]
    rr, rb = inputs.paint_droplets(shape, drops, periodic=(True, False, False))
    kw = dict(wall_y=1, wall_z=1, wall_u=0.02, sigma=0.02, beta=0.7, A_nc=0.02, h_min=3.0)
    fo, fg, _, _ = run_pair(lbm, shape, (rr, rb), 100, **kw)
    assert_parity(fo, fg)


def test_sliding_walls_couette_and_fp16(lbm):
    # single-fluid Couette flow reaches the linear profile; FP16 deviation storage of
    # a sheared two-layer state stays within 1e-3 of the oracle in rho
    ny, U = 16, 0.01
    shape = (4, ny, 8)
    g = lbm.Lattice(lbm.make_params(8, ny, 4, wall_y=1, wall_u=U))
    g.set_fields(np.ones(shape), np.zeros(shape))
    g.step(4000)
    want = U * (2 * (np.arange(ny) + 0.5) / ny - 1)
    # FP32 arithmetic over 4000 steps: within 3e-5 of U (the FP64 oracle is exact)
    assert np.abs(g.get_fields()["u"][0] - want[None, :, None]).max() < 3e-5 * U
    g.close()
    yy = np.arange(ny)[None, :, None] * np.ones(shape)
    rr = np.where(yy < ny / 2, 1.0, 0.0)
    kw = dict(wall_y=1, wall_u=U, sigma=0.01, beta=0.7)
    fo, fg, _, _ = run_pair(lbm, shape, (rr, 1.0 - rr), 200, storage="fp16", **kw)
    e = errs(fo, fg)
    assert e["rho_r"] <= 1e-3 and e["rho_b"] <= 1e-3, e


def _sc_pair(lbm, shape, drops, steps, storage="fp32", periodic=(True, True, True), **kw):
    rr, rb = inputs.paint_droplets(shape, drops, periodic=periodic)
    # a little of each species everywhere, as in a separated Shan-Chen mixture
    rr, rb = 0.96 * rr + 0.02, 0.96 * rb + 0.02
    return run_pair(lbm, shape, (rr, rb), steps, storage=storage, model="shan_chen", **kw)


def test_shan_chen_droplet_periodic(lbm):
    fo, fg, _, _ = _sc_pair(lbm, (32, 32, 32), [(16.0, 16.0, 16.0, 8.0)], 100, G_sc=1.6)
    assert_parity(fo, fg)


def test_shan_chen_walls_sliding_forces_unequal_tau(lbm):
    # ragged tiles, walls in y (sliding) and z, body force, unequal relaxation times
    shape = (14, 30, 50)
    drops = [(14.0, 12.0, 7.0, 5.5), (31.0, 17.0, 6.5, 5.0)]
    fo, fg, _, _ = _sc_pair(lbm, shape, drops, 100, periodic=(True, False, False), G_sc=1.4,
                            wall_y=1, wall_z=1, wall_u=0.01, tau_r=0.9, tau_b=1.2,
                            g=(2e-5, 0, 1e-5))
    assert_parity(fo, fg)


def test_shan_chen_chain_mode_and_fp16(lbm):
    # 150 x 60 x 64 runs the step kernel in chain mode (CTAs crossing tiles)
    shape = (64, 60, 150)
    drops = [(20.0, 12.0, 30.0, 6.0), (50.0, 30.0, 50.0, 7.0), (110.0, 40.0, 20.0, 8.0)]
    fo, fg, _, _ = _sc_pair(lbm, shape, drops, 20, periodic=(True, False, False), G_sc=1.5,
                            wall_y=1, wall_z=1)
    assert_parity(fo, fg)
    fo, fg, _, _ = _sc_pair(lbm, (24, 24, 24), [(12.0, 12.0, 12.0, 6.0)], 100, storage="fp16",
                            G_sc=1.6)
    e = errs(fo, fg)
    assert e["rho_r"] <= 1e-3 and e["rho_b"] <= 1e-3, e


def test_near_contact_field_matches_oracle_on_dense_emulsion(lbm):
    # A dense emulsion has many films thinner than h_cut. The GPU measures A_h with a
    # bounded ray march (it stops after the last sample that may be positive); the
    # oracle marches every ray in full. Same colour field, every node compared.
    n = 40
    w = inputs.dense_emulsion(L=n, volume_fraction=0.3, r_range=(4.0, 7.0), seed=11)
    g = lbm.Lattice(lbm.make_params(n, n, n, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    g.step(10)
    _, _, lag = g.get_pops()
    got = g.get_nc_field()
    op = oracle.make_params(n, n, n, **w.params)
    want = np.zeros_like(got)
    for z in range(n):
        for y in range(n):
            for x in range(n):
                want[z, y, x] = oracle.nc_strength_node(op, lag, x, y, z)
    # FP32 ray positions and interpolation locate a crossing to ~1e-5 lattice units,
    # which moves A_h by up to ~1e-4 of its value on the h^-3 tail
    A = w.params["A_nc"]
    tol = 1e-6 * A + 1e-3 * np.abs(want)
    bad = np.argwhere(np.abs(got - want) > tol)
    # every node beyond that must be a threshold branch: the oracle with the sign band
    # or the gradient threshold moved by its FP32 rounding bound gives the GPU's A_h
    unexplained = [(z, y, x) for z, y, x in bad
                   if not branch_cases.ah_explained(op, lag, x, y, z, got[z, y, x],
                                                    1e-6 * A + 1e-3 * abs(got[z, y, x]))]
    print("nodes with A_h > 0:", int((want > 0).sum()), "threshold branches:", len(bad))
    assert (want > 0).sum() > 200
    assert not unexplained, unexplained[:10]
    assert len(bad) <= max(2, int(1e-4 * want.size)), bad[:10]


@pytest.mark.parametrize("case", ["periodic", "walls"])
def test_near_contact_field_tensor_copied_cubes(lbm, case):
    # Lattices large enough that the near-contact pass copies the inner blocks' halo
    # cubes with one tensor copy (a 16 x 8 x 8 block whose 40 x 26 x 26 cube lies
    # inside the lattice; on walled axes the cube may reach past the walls) and the
    # others with element copies wrapped across the periodic seams: every node's A_h
    # against the oracle's full ray march, threshold branches proven as above.
    nz, ny, nx = (40, 48, 64) if case == "periodic" else (42, 34, 64)
    drops = inputs.dense_emulsion(L=64, volume_fraction=0.3, r_range=(4.0, 7.0), seed=12).droplets
    per = (True, True, True) if case == "periodic" else (True, False, False)
    drops = [d for d in drops if d[1] < ny - 2 and d[2] < nz - 2]
    rr, rb = inputs.paint_droplets((nz, ny, nx), drops, periodic=per)
    kw = dict(sigma=0.01, A_nc=0.01, h_min=3.0, kolmogorov_amp=1e-5)
    if case == "walls":
        kw.update(wall_y=1, wall_z=1)
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, **kw))
    g.set_fields(rr, rb)
    g.step(8)
    _, _, lag = g.get_pops()
    got = g.get_nc_field()
    op = oracle.make_params(nx, ny, nz, **kw)
    want = np.zeros_like(got)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                want[z, y, x] = oracle.nc_strength_node(op, lag, x, y, z)
    A = kw["A_nc"]
    bad = np.argwhere(np.abs(got - want) > 1e-6 * A + 1e-3 * np.abs(want))
    unexplained = [(z, y, x) for z, y, x in bad
                   if not branch_cases.ah_explained(op, lag, x, y, z, got[z, y, x],
                                                    1e-6 * A + 1e-3 * abs(got[z, y, x]))]
    print(case, "nodes with A_h > 0:", int((want > 0).sum()), "threshold branches:", len(bad))
    assert (want > 0).sum() > 200
    assert not unexplained, unexplained[:10]


def test_dense_emulsion_near_contact_30_steps(lbm):
    n = 40
    w = inputs.dense_emulsion(L=n, volume_fraction=0.3, r_range=(4.0, 7.0), seed=11)
    fo, fg, _, _ = run_pair(lbm, w.shape, (w.rho_r, w.rho_b), 30, **w.params)
    assert_parity(fo, fg)


def test_gel_quench_one_step_sampled(lbm):
    # Symmetric mixture with colour noise and 2 % pinning sites (the gel workload at
    # 48^3): after 20 GPU steps, one more step against the oracle evaluated at
    # sampled nodes from the same state.
    w = inputs.bicontinuous(L=48, seed=5)
    n = 48
    g = lbm.Lattice(lbm.make_params(n, n, n, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    g.set_pin_mask(w.pins)
    g.step(20)
    fr, fb, lag = g.get_pops()
    ah_gpu = g.get_nc_field().ravel()      # A_h the next step measures
    g.step(1)
    gr, gb, _ = g.get_pops()
    m = _map_to_oracle(lbm)
    N = n ** 3
    nodes = np.random.default_rng(4).choice(N, 3000, replace=False)
    P = oracle.make_params(n, n, n, **w.params)
    fro, fbo, pins = fr.reshape(19, N)[m], fb.reshape(19, N)[m], w.pins.ravel()
    oa, ob, _ = oracle.step_nodes(P, fro, fbo, lag.ravel(), nodes, pin=pins)
    ga = gr.reshape(19, N)[m][:, nodes].T
    gbb = gb.reshape(19, N)[m][:, nodes].T
    bad = np.nonzero((np.abs(oa - ga).max(1) > 1e-6) | (np.abs(ob - gbb).max(1) > 1e-6))[0]
    # a node whose film measurement has a sample (or whose lagged gradient lies)
    # within FP32 rounding of a threshold may take the other branch in FP32: each
    # such node must be reproduced by the oracle with that threshold moved by its
    # rounding bound; any other difference fails
    unexplained = [int(nodes[k]) for k in bad
                   if not branch_cases.step_explained(P, fro, fbo, lag.ravel(), int(nodes[k]),
                                                      ga[k], gbb[k], ah_gpu[nodes[k]], pin=pins)]
    print("sampled nodes:", len(nodes), "threshold branches:", len(bad))
    assert not unexplained, (unexplained[:10], np.abs(oa - ga).max())


def test_zero_steps_returns_set_fields(lbm):
    shape = (5, 6, 7)
    rr, rb, u = inputs.random_state(shape, seed=3)
    g = lbm.Lattice(lbm.make_params(7, 6, 5))
    g.set_fields(rr, rb, u)
    g.step(0)
    f = g.get_fields()
    assert np.abs(f["rho_r"] - rr).max() < 2e-7 and np.abs(f["rho_b"] - rb).max() < 2e-7
    assert np.abs(f["u"] - u).max() < 1e-7


def test_conservation_on_gpu(lbm):
    w = inputs.static_droplet(L=32, R=8.0)
    g = lbm.Lattice(lbm.make_params(32, 32, 32, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    t0 = g.observables()
    g.step(500)
    t = g.observables()
    # FP32 arithmetic: per-species mass conserved to FP32 round-off accumulation
    assert abs(t[0] - t0[0]) / t0[0] < 1e-6 and abs(t[1] - t0[1]) / t0[1] < 1e-6
    assert np.abs(t[2:5]).max() / (t0[0] + t0[1]) < 1e-7
    assert t[5] == 500


def test_laplace_on_gpu_matches_oracle(lbm):
    w = inputs.static_droplet(L=32, R=8.0)
    fo, fg, o, g = run_pair(lbm, w.shape, (w.rho_r, w.rho_b), 200, **w.params)
    lo = o.laplace((16, 16, 16))
    lg = g.laplace((16, 16, 16))
    assert abs(lg["R_eff"] - lo["R_eff"]) < 1e-4
    assert abs(lg["dp"] - lo["dp"]) / abs(lo["dp"]) < 1e-3


def test_checkpoint_resume_is_bitwise(lbm):
    w = inputs.channel_droplets(nx=64, ny=40, nz=24, n_grid=(2, 2, 1), r_range=(4, 6), seed=5)
    P = lbm.make_params(64, 40, 24, **w.params)
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
    assert b.steps_taken == 60


def test_fp16_deviation_storage_accuracy(lbm):
    w = inputs.static_droplet(L=32, R=8.0)
    fo, fg, o, g = run_pair(lbm, w.shape, (w.rho_r, w.rho_b), 100, storage="fp16", **w.params)
    e = errs(fo, fg)
    print("fp16 static droplet, 100 steps:", e)
    assert e["rho_r"] <= 1e-3 and e["rho_b"] <= 1e-3, e


def test_fp16_deviation_storage_walls_and_near_contact(lbm):
    # bounce-back links and periodic ghosts decode against the colour field of
    # their source node (own node for a bounced link)
    w = inputs.channel_droplets(nx=64, ny=40, nz=24, n_grid=(2, 2, 1), r_range=(4, 6), seed=5)
    fo, fg, _, _ = run_pair(lbm, w.shape, (w.rho_r, w.rho_b), 100, storage="fp16", **w.params)
    e = errs(fo, fg)
    print("fp16 channel, 100 steps:", e)
    assert e["rho_r"] <= 1e-3 and e["rho_b"] <= 1e-3, e


def test_fp16_deviation_storage_laplace_pressure_jump(lbm):
    w = inputs.static_droplet(L=32, R=8.0)
    fo, fg, o, g = run_pair(lbm, w.shape, (w.rho_r, w.rho_b), 200, storage="fp16", **w.params)
    lo = o.laplace((16, 16, 16))
    lg = g.laplace((16, 16, 16))
    print("fp16 Laplace dp:", lg["dp"], "oracle:", lo["dp"])
    assert abs(lg["dp"] - lo["dp"]) / abs(lo["dp"]) < 0.02


def test_bf16_deviation_storage_accuracy(lbm):
    # BF16 keeps 8 mantissa bits; with the colour-split reference the stored
    # deviations are small enough for it to hold the FP16 density bar as well
    w = inputs.static_droplet(L=32, R=8.0)
    fo, fg, o, g = run_pair(lbm, w.shape, (w.rho_r, w.rho_b), 100, storage="bf16", **w.params)
    e = errs(fo, fg)
    print("bf16 static droplet, 100 steps:", e)
    assert all(math.isfinite(v) for v in e.values()), e
    assert e["rho_r"] <= 1e-3 and e["rho_b"] <= 1e-3, e


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_deviation_storage_pops_round_trip(lbm, storage):
    # get_pops decodes against the current colour field and set_pops re-encodes
    # against the one it is given: the state survives the round trip
    w = inputs.channel_droplets(nx=64, ny=40, nz=24, n_grid=(2, 2, 1), r_range=(4, 6), seed=5)
    P = lbm.make_params(64, 40, 24, storage=storage, **w.params)
    a = lbm.Lattice(P)
    a.set_fields(w.rho_r, w.rho_b)
    a.step(10)
    fr, fb, lag = a.get_pops()
    b = lbm.Lattice(P)
    b.set_fields(w.rho_r, w.rho_b)
    b.set_pops(fr, fb, lag)
    fr2, fb2, lag2 = b.get_pops()
    assert np.array_equal(lag, lag2)
    assert np.abs(fr2 - fr).max() <= 1e-6 and np.abs(fb2 - fb).max() <= 1e-6


def test_window_matches_full_download_with_wrap(lbm):
    # a box that wraps around all three periodic axes, against the full download
    shape = (12, 10, 16)
    rr, rb, u = inputs.random_state(shape, seed=8, u_amp=0.01)
    for storage in ("fp32", "fp16"):
        g = lbm.Lattice(lbm.make_params(16, 10, 12, sigma=0.01, storage=storage))
        g.set_fields(rr, rb, u)
        g.step(3)
        fr, fb, lag = g.get_pops()
        x0, y0, z0, wx, wy, wz = 13, -2, 9, 7, 5, 6
        wr, wb, wl = g.get_window(x0, y0, z0, wx, wy, wz)
        zz = (np.arange(z0, z0 + wz) % 12)[:, None, None]
        yy = (np.arange(y0, y0 + wy) % 10)[None, :, None]
        xx = (np.arange(x0, x0 + wx) % 16)[None, None, :]
        assert np.array_equal(wr, fr[:, zz, yy, xx]) and np.array_equal(wb, fb[:, zz, yy, xx])
        assert np.array_equal(wl, lag[zz, yy, xx])
    with pytest.raises(lbm.LbmError):
        g.get_window(0, 0, 0, 17, 1, 1)


def test_invalid_arguments_are_rejected(lbm):
    for bad in (dict(tau_r=0.5), dict(beta=1.5), dict(storage=7), dict(wall_u=0.01),
                dict(model=5), dict(model="shan_chen", A_nc=0.01), dict(wall_y=1, wall_u=0.5)):
        kw = dict(tau_r=1.0)
        kw.update(bad)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.Lattice(lbm.make_params(8, 8, 8, **kw))
        assert ei.value.status == -1
    g = lbm.Lattice(lbm.make_params(8, 8, 8))
    with pytest.raises(lbm.LbmError) as ei:
        g.step(1)                     # no fields yet
    assert ei.value.status == -4
    with pytest.raises(lbm.LbmError):
        g.step(-1)


def _map_to_oracle(lbm):
    """index map: oracle direction k -> library direction."""
    cg = lbm.velocity_set()
    co = oracle.lattice()[0]
    return np.array([int(np.nonzero((cg == co[k]).all(1))[0][0]) for k in range(19)])


def test_one_step_full_size_channel_sampled(lbm):
    # The microfluidic-crystal channel at its full size (256 x 128 x 64, 40 droplets)
    # after 50 GPU steps: one more GPU step compared with the oracle's step evaluated
    # at 4000 sampled nodes from the same (downloaded) state.
    w = inputs.channel_droplets()
    nz, ny, nx = w.shape
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    g.step(50)
    fr, fb, lag = g.get_pops()
    g.step(1)
    gr, gb, _ = g.get_pops()
    m = _map_to_oracle(lbm)
    N = nx * ny * nz
    frr = fr.reshape(19, N)[m]
    fbb = fb.reshape(19, N)[m]
    rng = np.random.default_rng(9)
    phi = lag.ravel()
    iface = np.nonzero(np.abs(phi) < 0.9)[0]
    nodes = np.unique(np.concatenate([rng.choice(N, 2000, replace=False),
                                      rng.choice(iface, 2000, replace=False)]))
    P = oracle.make_params(nx, ny, nz, **w.params)
    oa, ob, _ = oracle.step_nodes(P, frr, fbb, phi, nodes)
    ga = gr.reshape(19, N)[m][:, nodes].T
    gbb = gb.reshape(19, N)[m][:, nodes].T
    assert np.abs(oa - ga).max() < 1e-6 and np.abs(ob - gbb).max() < 1e-6


def test_bounded_wait_gives_up_and_the_context_stays_usable(lbm):
    # failure detection without a GPU fault: a wait that cannot complete times out,
    # the host reads LBM_ETIMEOUT, and the same context then steps as if nothing
    # had happened
    shape = (16, 16, 32)
    rr, rb = inputs.paint_droplets(shape, [(16.0, 8.0, 8.0, 5.0)])
    a = lbm.Lattice(lbm.make_params(32, 16, 16, sigma=0.01))
    b = lbm.Lattice(lbm.make_params(32, 16, 16, sigma=0.01))
    for g in (a, b):
        g.set_fields(rr, rb)
        g.step(5)
    assert a.selftest_timeout() == -5
    for g in (a, b):
        g.step(5)
    fa, fb = a.get_pops(), b.get_pops()
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(fa[1], fb[1])
    a.close()
    b.close()


def test_mapped_host_buffers_equal_staged_ones(lbm):
    # Pinned host buffers mapped into the device's address space are read and written by
    # the kernels directly; pageable (NumPy) ones go through the staging buffer. Both
    # give the same bits, and reading the fields mid-run (which re-measures A_h into the
    # A_h buffer) leaves the run unchanged.
    torch = pytest.importorskip("torch")
    shape = (24, 40, 64)
    nz, ny, nx = shape
    drops = [(20.0, 20.0, 12.0, 7.0), (36.0, 20.0, 12.0, 7.5)]
    rr, rb = inputs.paint_droplets(shape, drops)
    _, _, u = inputs.random_state(shape, seed=8, u_amp=0.005)
    kw = dict(sigma=0.02, beta=0.7, A_nc=0.02, h_min=3.0, kolmogorov_amp=1e-4)
    a = lbm.Lattice(lbm.make_params(nx, ny, nz, **kw))
    b = lbm.Lattice(lbm.make_params(nx, ny, nz, **kw))
    c = lbm.Lattice(lbm.make_params(nx, ny, nz, **kw))
    pin = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()
    a.set_fields(rr, rb, u)
    b.set_fields(pin(rr), pin(rb), pin(u))
    c.set_fields(rr, rb, u)
    assert all(np.array_equal(x, y) for x, y in zip(a.get_pops(), b.get_pops()))
    for g in (a, b, c):
        g.step(5)
    fa = a.get_fields()
    outs = {"rho_r": torch.empty(shape, dtype=torch.float64).pin_memory(),
            "rho_b": torch.empty(shape, dtype=torch.float64).pin_memory(),
            "u": torch.empty((3,) + shape, dtype=torch.float64).pin_memory(),
            "phi": torch.empty(shape, dtype=torch.float64).pin_memory()}
    b.get_fields(outs)
    for k in fa:
        assert np.array_equal(fa[k], outs[k].numpy()), k
    for g in (a, b, c):
        g.step(3)
    pa, pb, pc = a.get_pops(), b.get_pops(), c.get_pops()
    assert all(np.array_equal(x, y) for x, y in zip(pa, pc))
    assert all(np.array_equal(x, y) for x, y in zip(pb, pc))
    for g in (a, b, c):
        g.close()
