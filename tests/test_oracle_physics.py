"""Pins of the FP64 oracle's whole step: exact streaming, conservation, momentum
balance, Poiseuille flow, the Laplace law, near-contact merging behaviour, and
symmetries. Thresholds are the ones the method fixes (conservation to round-off,
Poiseuille within 1 %, Laplace within 3 %), except where a measured limit of the
discretisation is stated beside the check.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mini
from paper_2005_12764_gb300 import inputs

C, W, OPP, B = oracle.lattice()


def _lattice(shape, fields=None, **kw):
    nz, ny, nx = shape
    lat = oracle.Lattice(oracle.make_params(nx, ny, nz, **kw))
    if fields is not None:
        lat.set_fields(*fields)
    return lat


# ------------------------------------------------------------------ streaming
def test_streaming_is_exact_permutation_periodic():
    # streaming alone for lcm(nx, ny, nz) steps returns every population bitwise
    shape = (5, 3, 4)
    lat = _lattice(shape)
    r = np.random.default_rng(1)
    fr, fb = r.random((19,) + shape), r.random((19,) + shape)
    lat.set_pops(fr, fb)
    lat.stream_only(1)
    gr, gb = lat.get_pops()
    for i in range(19):        # one step equals a periodic shift by c_i (brute force)
        want = np.roll(fr[i], shift=(C[i][2], C[i][1], C[i][0]), axis=(0, 1, 2))
        assert np.array_equal(gr[i], want)
    lat.stream_only(60 - 1)
    gr, gb = lat.get_pops()
    assert np.array_equal(gr, fr) and np.array_equal(gb, fb)


def test_streaming_with_walls_is_exact_permutation():
    # halfway bounce-back keeps streaming a permutation: period lcm(nx, 2 ny, 2 nz)
    shape = (5, 3, 4)
    lat = _lattice(shape, wall_y=1, wall_z=1)
    r = np.random.default_rng(2)
    fr, fb = r.random((19,) + shape), r.random((19,) + shape)
    lat.set_pops(fr, fb)
    lat.stream_only(1)
    gr, _ = lat.get_pops()
    assert np.array_equal(np.sort(gr.ravel()), np.sort(fr.ravel()))
    # a population at y = 0 moving towards the wall comes back reversed, in place
    i_down = [i for i in range(19) if tuple(C[i]) == (0, -1, 0)][0]
    i_up = OPP[i_down]
    assert np.array_equal(gr[i_up][:, 0, :], fr[i_down][:, 0, :])
    lat.stream_only(60 - 1)
    gr, gb = lat.get_pops()
    assert np.array_equal(gr, fr) and np.array_equal(gb, fb)


# ------------------------------------------------------------------ conservation
def test_conservation_static_droplet_500_steps():
    w = inputs.static_droplet(L=32, R=8.0)
    lat = _lattice(w.shape, (w.rho_r, w.rho_b), **w.params)
    t0 = lat.totals()
    lat.step(500)
    t = lat.totals()
    M = t0[0] + t0[1]
    assert abs(t[0] - t0[0]) / t0[0] < 1e-12
    assert abs(t[1] - t0[1]) / t0[1] < 1e-12
    assert np.abs(t[2:]).max() / M < 1e-12


def test_momentum_changes_by_total_force():
    # periodic box, body + Kolmogorov + near-contact forces: P(t+1) - P(t) = sum_x F
    shape = (16, 16, 24)
    drops = [(7.0, 8.0, 8.0, 5.0), (17.0, 8.0, 8.0, 5.0)]
    rr, rb = inputs.paint_droplets(shape, drops)
    lat = _lattice(shape, (rr, rb), sigma=0.01, A_nc=0.05, g=(2e-5, -1e-5, 3e-6),
                   kolmogorov_amp=1e-4)
    P0 = lat.totals()[2:]
    nc_seen = 0.0
    for _ in range(20):
        lat.step(1)
        P1 = lat.totals()[2:]
        F = lat.get_forces()
        dP = F.reshape(3, -1).sum(1)
        assert np.allclose(P1 - P0, dP, rtol=0, atol=1e-13)
        body = np.array([2e-5, -1e-5, 3e-6]) * rr.size
        nc_seen = max(nc_seen, np.abs(dP - body).max())
        P0 = P1
    assert nc_seen > 1e-6     # the near-contact force did act and is balanced too


# ------------------------------------------------------------------ Poiseuille
def test_poiseuille_profile_within_one_percent():
    ny, g = 32, 1e-6
    shape = (2, ny, 2)
    lat = _lattice(shape, (np.ones(shape), np.zeros(shape)), wall_y=1, tau_r=1.0,
                   g=(g, 0, 0))
    lat.step(12000)
    u = lat.get_fields()["u"][0][0, :, 0]
    nu = (1.0 - 0.5) / 3
    y = np.arange(ny)
    exact = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(u - exact).max() / exact.max() < 0.01


# ------------------------------------------------------------------ sliding walls
@pytest.mark.parametrize("tau", [1.0, 0.8, 1.7])
def test_couette_between_sliding_walls_is_exact(tau):
    # walls at y = -1/2 (moving -U) and ny - 1/2 (+U) along x: the steady profile of
    # plain Couette flow, u_x = U (2 (y + 1/2)/ny - 1), is reached to round-off
    # (halfway bounce-back places a moving wall exactly for linear flow, any tau)
    ny, U = 12, 0.01
    shape = (3, ny, 4)
    lat = _lattice(shape, (np.ones(shape), np.zeros(shape)), wall_y=1, tau_r=tau, wall_u=U)
    lat.step(6000)
    f = lat.get_fields()
    want = U * (2 * (np.arange(ny) + 0.5) / ny - 1)
    assert np.abs(f["u"][0] - want[None, :, None]).max() < 1e-13
    assert np.abs(f["u"][1]).max() < 1e-13 and np.abs(f["u"][2]).max() < 1e-13


def test_sliding_walls_two_layers_conserve_mass_and_stay_linear():
    # red below y = ny/2, blue above, sheared by the walls: each species' mass is
    # conserved to round-off, the net x momentum stays zero (the set-up is invariant
    # under (x, y) -> (-x, ny-1-y)), and with equal viscosities the profile is the
    # single-fluid Couette profile
    nx, ny, nz, U = 6, 16, 4, 0.02
    shape = (nz, ny, nx)
    yy = np.arange(ny)[None, :, None] * np.ones(shape)
    rr = np.where(yy < ny / 2, 1.0, 0.0)
    lat = _lattice(shape, (rr, 1.0 - rr), wall_y=1, tau_r=1.0, sigma=0.01, beta=0.7, wall_u=U)
    m0 = lat.totals()
    lat.step(4000)
    m1 = lat.totals()
    f = lat.get_fields()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-12 and abs(m1[1] - m0[1]) / m0[1] < 1e-12
    assert abs(((f["rho_r"] + f["rho_b"]) * f["u"][0]).sum()) < 1e-12
    want = U * (2 * (np.arange(ny) + 0.5) / ny - 1)
    assert np.abs(f["u"][0] - want[None, :, None]).max() < 1e-12


def test_sliding_walls_at_rest_are_plain_bounce_back():
    shape = (6, 7, 5)
    rr, rb, u = inputs.random_state(shape, seed=3)
    kw = dict(wall_y=1, wall_z=1, sigma=0.02, beta=0.7, g=(1e-4, 0, 0))
    a = _lattice(shape, (rr, rb, u), **kw)
    b = _lattice(shape, (rr, rb, u), wall_u=0.0, **kw)
    c = _lattice(shape, (rr, rb, u), wall_u=0.01, **kw)
    for lat in (a, b, c):
        lat.step(5)
    pa, pb, pc = a.get_pops(), b.get_pops(), c.get_pops()
    assert all(np.array_equal(x, y) for x, y in zip(pa, pb))
    assert not np.array_equal(pa[0], pc[0])


# ------------------------------------------------------------------ Laplace law
def _laplace_ratio(L, R, steps):
    w = inputs.static_droplet(L=L, R=R)
    lat = _lattice(w.shape, (w.rho_r, w.rho_b), **w.params)
    lat.step(steps)
    lap = lat.laplace((L / 2, L / 2, L / 2))
    return lap["dp"] / (2 * w.params["sigma"] / lap["R_eff"]), lap


def test_laplace_static_droplet_R8_32cube():
    # The static-droplet workload itself: 32^3, R = 8, sigma = 0.01, 500 steps.
    # Measured: dp / (2 sigma / R_eff) = 1.042 at 500 steps (a damped pressure
    # oscillation), 1.0548 once relaxed. The excess over Laplace's law is the
    # finite interface width (~4 lu) against R = 8; the fit over R below removes it.
    ratio, lap = _laplace_ratio(32, 8.0, 500)
    assert abs(ratio - 1.0) < 0.06, lap
    assert 7.5 < lap["R_eff"] < 8.2


@pytest.mark.slow
def test_laplace_fit_over_R():
    # Laplace's law dp = 2 sigma / R pins the surface-tension constant of the
    # perturbation (sigma = 2 A / (9 omega)). Relaxed static droplets (L = 4R, run
    # until dp has settled to 1e-4) of R = 8, 10, 12 give dp R / (2 sigma) = 1.0548,
    # 1.0319, 1.0191: the excess falls as R^-2.4, the finite interface width against
    # R. A least-squares fit of dp R / (2 sigma) = s + c / R^2 takes that
    # discretisation term out; its R -> infinity limit s must be 1 within 3 % (a
    # factor-2 error in the constant gives 2 or 1/2). Measured s = 0.991.
    Rs, steps = (8.0, 10.0, 12.0), (2000, 2500, 3000)
    ratios, reff = [], []
    for R, n in zip(Rs, steps):
        ratio, lap = _laplace_ratio(int(4 * R), R, n)
        assert abs(lap["R_eff"] - R) < 0.1, lap
        ratios.append(ratio)
        reff.append(lap["R_eff"])
    Reff = np.array(reff)
    A = np.stack([np.ones(3), 1.0 / Reff ** 2], axis=1)
    (s_inf, c), *_ = np.linalg.lstsq(A, np.array(ratios), rcond=None)
    print("dp R / (2 sigma):", ratios, "fit: s =", s_inf, "c =", c)
    assert abs(s_inf - 1.0) < 0.03, (ratios, s_inf, c)
    assert c > 0 and ratios[0] > ratios[1] > ratios[2]       # the excess decays with R
    assert abs(ratios[2] - 1.0) < 0.03, ratios               # R = 12 already within 3 %


# ------------------------------------------------------------------ near contact
def _components(phi):
    from scipy import ndimage
    return ndimage.label(phi > 0)[1]


@pytest.mark.slow
@pytest.mark.parametrize("A_nc,expect", [(0.0, 1), (0.001, 1), (0.02, 1), (0.03, 2), (0.05, 2)])
def test_near_contact_inhibits_merging(A_nc, expect):
    # Two R = 8 droplets 2 lu apart (sigma = 0.01), capillary number N_c = A dx / sigma
    # (Eq. 11 and the paragraph after it: N_c << 1 merges, N_c ~ 1 inhibits merging).
    # Without the force (N_c = 0) and well below one (N_c = 0.1) the film drains and
    # the droplets merge; the film survives from N_c = 3 on (checked at 5 as well).
    # With this reading the transition lies between N_c = 2 (merges) and 3: the
    # repulsion per unit film area is integral A_h |G| dn = 2 A (phi spans -1 .. 1),
    # twice the A of a unit-weight delta function, and it competes with the
    # diffuse-interface attraction of two interfaces 2 lu apart, so the transition
    # sits at N_c of order one, a few units, as the paper's order-of-magnitude
    # statement has it.
    shape = (32, 32, 48)
    drops = [(14.0, 16.0, 16.0, 8.0), (34.0, 16.0, 16.0, 8.0)]
    rr, rb = inputs.paint_droplets(shape, drops)
    lat = _lattice(shape, (rr, rb), sigma=0.01, A_nc=A_nc, h_min=3.0)
    lat.step(500)
    assert _components(lat.get_fields()["phi"]) == expect


def test_near_contact_film_thickness_flat_films():
    # Brute force in 1-D: for a profile varying along x only, the ray samples a
    # piecewise-linear interpolant exactly, so h is the distance between its zeros.
    nx = 40
    x = np.arange(nx)
    prof = np.where((x >= 8) & (x < 16) | (x >= 16 + 4) & (x < 30), 1.0, -1.0)
    prof = np.convolve(np.pad(prof, 2, mode="wrap"), np.ones(3) / 3, mode="same")[2:-2]
    phi = np.broadcast_to(prof, (4, 4, nx)).copy()
    p = oracle.make_params(nx, 4, 4, A_nc=0.02, h_min=3.0, h_cut=6.0)
    G = oracle.gradient(p, phi)
    checked = 0
    for xi in range(nx):
        g = G[:, 1, 1, xi]
        if np.linalg.norm(g) < 1e-3:
            continue
        F = oracle.nc_strength_node(p, phi, xi, 1, 1) * g
        s = -np.sign(g[0])                        # ray direction along x
        ts = -1 + 0.5 * np.arange(19)
        vals = np.interp((xi + s * ts) % nx, np.arange(nx + 1), np.append(prof, prof[0]))
        zs = []
        for k in range(len(ts) - 1):
            v0, v1 = vals[k], vals[k + 1]
            if (not zs and v0 > 0 >= v1) or (zs and v0 <= 0 < v1):
                zs.append(ts[k] + 0.5 * v0 / (v0 - v1))
                if len(zs) == 2:
                    break
        want = oracle.A_h(zs[1] - zs[0], 0.02, 3.0, 6.0) * g if len(zs) == 2 else 0 * g
        assert np.allclose(F, want, atol=1e-15)
        checked += int(len(zs) == 2 and np.abs(want).max() > 0)
    assert checked >= 4


def test_near_contact_strength_oblique_rays_brute_force():
    # Brute force in 3-D: two smooth droplets (phi = tanh((R - r)/1.5), periodic) on an
    # oblique line, so the rays run between lattice directions. At every node with
    # |G| >= 1e-3 the strength must equal the reading restated here with an
    # independent trilinear sampler (scipy's map_coordinates, periodic): samples at
    # x - t G/|G|, t = -1, -1/2, ..., h_cut + 2; samples with |phi| <= 1e-5 unsigned;
    # h between the first downward and the next upward crossing, each located
    # linearly between consecutive signed samples; A_h(h) of Eq. 11, else 0.
    from scipy.ndimage import map_coordinates
    nz, ny, nx = 24, 26, 36
    drops = [(11.0, 12.3, 11.6, 5.0), (24.2, 14.1, 13.0, 5.5)]     # gap ~2.9 lu
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    phi = -np.ones((nz, ny, nx))
    for cx, cy, cz, R in drops:
        d = [((a - c + n / 2) % n) - n / 2 for a, c, n in ((xx, cx, nx), (yy, cy, ny), (zz, cz, nz))]
        phi = np.maximum(phi, np.tanh((R - np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)) / 1.5))
    A, hmin, hcut = 0.02, 3.0, 6.0
    p = oracle.make_params(nx, ny, nz, A_nc=A, h_min=hmin, h_cut=hcut)
    G = oracle.gradient(p, phi)
    gm = np.sqrt((G * G).sum(0))
    ts = -1.0 + 0.5 * np.arange(int(np.floor(2 * (hcut + 3))) + 1)
    checked = films = 0
    for z, y, x in zip(*np.nonzero(gm >= 1e-3)):
        n = -G[:, z, y, x] / gm[z, y, x]
        coords = np.array([z + ts * n[2], y + ts * n[1], x + ts * n[0]])
        vals = map_coordinates(phi, coords, order=1, mode="grid-wrap")
        signed = [(t, v) for t, v in zip(ts, vals) if abs(v) > 1e-5]
        t_d = t_u = None
        for (t0, v0), (t1, v1) in zip(signed, signed[1:]):
            if t_d is None and v0 > 0 > v1:
                t_d = t0 + (t1 - t0) * v0 / (v0 - v1)
            elif t_d is not None and v0 < 0 < v1:
                t_u = t0 + (t1 - t0) * v0 / (v0 - v1)
                break
        want = oracle.A_h(t_u - t_d, A, hmin, hcut) if t_u is not None else 0.0
        got = oracle.nc_strength_node(p, phi, int(x), int(y), int(z))
        assert abs(got - want) <= 1e-12, (x, y, z, got, want)
        checked += 1
        films += want > 0
    assert checked > 1000 and films >= 20, (checked, films)


# ------------------------------------------------------------------ symmetries
@pytest.mark.parametrize("A_nc", [0.0, 0.01])
def test_translation_invariance(A_nc):
    # Shifting the initial state by a lattice vector shifts the result: bitwise
    # without the near-contact force; with it, the ray's sample points x + t n round
    # differently at different x, so agreement is to round-off.
    shape = (10, 9, 12)
    rr, rb, u = inputs.random_state(shape, seed=11)
    kw = dict(sigma=0.02, A_nc=A_nc, g=(1e-5, 0, 0), tau_r=0.9, tau_b=1.2)
    a = _lattice(shape, (rr, rb, u), **kw)
    a.step(6)
    s = (3, 0, 5)   # shift in (z, y, x); y kept because nothing here depends on y
    roll = lambda f: np.roll(f, s, axis=(-3, -2, -1))
    b = _lattice(shape, (roll(rr), roll(rb), roll(u)), **kw)
    b.step(6)
    fa, fb_ = a.get_pops(), b.get_pops()
    if A_nc == 0.0:
        assert np.array_equal(roll(fa[0]), fb_[0]) and np.array_equal(roll(fa[1]), fb_[1])
    else:
        assert np.allclose(roll(fa[0]), fb_[0], rtol=0, atol=1e-14)
        assert np.allclose(roll(fa[1]), fb_[1], rtol=0, atol=1e-14)


def test_mirror_symmetry_x():
    shape = (8, 9, 10)
    rr, rb, u = inputs.random_state(shape, seed=12)
    kw = dict(sigma=0.02, A_nc=0.01, wall_y=1)
    a = _lattice(shape, (rr, rb, u), **kw)
    a.step(5)
    mir = lambda f: np.roll(f[..., ::-1], 1, axis=-1)   # x -> -x (mod nx)
    um = np.stack([-mir(u[0]), mir(u[1]), mir(u[2])])
    b = _lattice(shape, (mir(rr), mir(rb), um), **kw)
    b.step(5)
    fa, fb_ = a.get_fields(), b.get_fields()
    assert np.allclose(mir(fa["rho_r"]), fb_["rho_r"], atol=1e-14)
    assert np.allclose(-mir(fa["u"][0]), fb_["u"][0], atol=1e-15)
    assert np.allclose(mir(fa["u"][1]), fb_["u"][1], atol=1e-15)


# ------------------------------------------------------------------ cross-checks
@pytest.mark.parametrize("case", [
    dict(shape=(4, 4, 4)),
    dict(shape=(5, 6, 7), wall_y=1, g=(1e-4, 2e-5, 0), tau_b=1.3),
    dict(shape=(8, 6, 7), wall_z=1, wall_y=1, A_nc=0.02, kolmogorov_amp=1e-3, tau_r=0.8),
    dict(shape=(8, 8, 8), A_nc=0.05, h_min=2.0),
    dict(shape=(6, 7, 5), wall_y=1, wall_z=1, wall_u=0.03, A_nc=0.02, tau_b=0.9),
])
def test_numpy_mini_oracle_agrees(case):
    case = dict(case)
    shape = case.pop("shape")
    nz, ny, nx = shape
    rr, rb, u = inputs.random_state(shape, seed=sum(shape))
    kw = dict(sigma=0.02, beta=0.7, **case)
    lat = _lattice(shape, (rr, rb, u), **kw)
    m = mini.MiniLattice(nx, ny, nz, **kw)
    m.set_fields(rr, rb, u)
    lat.step(4)
    m.step(4)
    f = lat.get_fields()
    for k in ("rho_r", "rho_b", "phi"):
        assert np.allclose(f[k], m.last[k], rtol=0, atol=1e-13), k
    assert np.allclose(f["u"], m.last["u"], rtol=0, atol=1e-13)
    assert np.allclose(lat.get_forces(), m.last["F"], rtol=0, atol=1e-13)


def test_step_nodes_matches_full_step():
    w = inputs.channel_droplets(nx=64, ny=40, nz=24, n_grid=(2, 2, 1), r_range=(4, 6),
                                seed=5)
    shape = w.shape
    lat = _lattice(shape, (w.rho_r, w.rho_b), **w.params)
    lat.step(3)
    fr, fb = lat.get_pops()
    lag = lat.get_phi_lag()
    nodes = np.random.default_rng(3).choice(fr[0].size, 300, replace=False)
    lat.step(1)
    gr, gb = lat.get_pops()
    p = oracle.make_params(shape[2], shape[1], shape[0], **w.params)
    oa, ob, F = oracle.step_nodes(p, fr.reshape(19, -1), fb.reshape(19, -1), lag.ravel(), nodes)
    assert np.array_equal(oa, gr.reshape(19, -1)[:, nodes].T)
    assert np.array_equal(ob, gb.reshape(19, -1)[:, nodes].T)


def test_near_contact_with_the_gradient_given_is_the_same_strength():
    # the oracle entry that takes the lagged gradient as given (used to bound the FP32
    # rounding of the ray direction) returns the pinned strength when given the node's
    # own gradient, and moves continuously with it
    from paper_2005_12764_gb300 import inputs
    shape = (12, 16, 24)
    rr, rb = inputs.paint_droplets(shape, [(7.0, 8.0, 6.0, 4.5), (16.5, 8.0, 6.0, 4.5)])
    phi = (rr - rb) / (rr + rb)
    P = oracle.make_params(24, 16, 12, A_nc=0.02, h_min=3.0)
    G = oracle.gradient(P, phi)
    seen = 0
    for (z, y, x) in [(6, 8, 11), (6, 8, 12), (6, 8, 10), (5, 7, 11), (6, 9, 13), (2, 2, 2)]:
        want = oracle.nc_strength_node(P, phi, x, y, z)
        assert oracle.nc_strength_node_g(P, phi, x, y, z, G[:, z, y, x]) == want
        near = oracle.nc_strength_node_g(P, phi, x, y, z, G[:, z, y, x] * (1 + 1e-9))
        assert abs(near - want) <= 1e-6 * max(1e-3, abs(want))
        seen += want > 0
    assert seen >= 2
