"""Pins of the FP64 oracle's per-node routines against closed forms and invariants.

Each check is derived from the mathematics of the method (moments of the D3Q19
set, Eqs. (1)-(9) of the paper, and the readings for the colour-gradient steps),
not by re-evaluating the oracle's own formula.
"""
import itertools
import math

import numpy as np
import pytest

import oracle

C, W, OPP, B = oracle.lattice()
Cf = C.astype(float)
rng = np.random.default_rng(7)


def moments(f):
    return f.sum(), Cf.T @ f, np.einsum("ia,ib,i->ab", Cf, Cf, f)


# ------------------------------------------------------------------ lattice tables
def test_velocity_set_is_d3q19():
    # brute force: the vectors of {-1,0,1}^3 with |c|^2 <= 2 (rest, 6 faces, 12 edges)
    want = {v for v in itertools.product((-1, 0, 1), repeat=3) if sum(a * a for a in v) <= 2}
    got = {tuple(int(a) for a in c) for c in C}
    assert len(got) == 19 and got == want


def test_weights_isotropy():
    assert math.isclose(W.sum(), 1.0, rel_tol=0, abs_tol=1e-15)
    I = np.eye(3)
    assert np.allclose(np.einsum("i,ia->a", W, Cf), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", W, Cf, Cf), I / 3, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", W, Cf, Cf, Cf), 0, atol=1e-16)
    four = np.einsum("i,ia,ib,ic,id->abcd", W, Cf, Cf, Cf, Cf)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) / 9
    assert np.allclose(four, iso, atol=1e-16)


def test_opposite_index():
    for i in range(19):
        assert (C[OPP[i]] == -C[i]).all()


# ------------------------------------------------------------------ equilibrium Eq. (2)
@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(seed):
    r = np.random.default_rng(seed)
    rho = r.uniform(0.2, 2.0)
    u = r.uniform(-0.1, 0.1, 3)
    m0, m1, m2 = moments(oracle.feq(rho, u))
    assert abs(m0 - rho) <= 1e-15 * rho * 4
    assert np.allclose(m1, rho * u, rtol=0, atol=1e-16)
    assert np.allclose(m2, rho * (np.eye(3) / 3 + np.outer(u, u)), rtol=0, atol=1e-15)
    # third moment (linear part): rho/3 (u_a d_bc + u_b d_ac + u_c d_ab), exact on D3Q19
    m3 = np.einsum("ia,ib,ic,i->abc", Cf, Cf, Cf, oracle.feq(rho, u))
    I = np.eye(3)
    want = rho / 3 * (np.einsum("a,bc->abc", u, I) + np.einsum("b,ac->abc", u, I)
                      + np.einsum("c,ab->abc", u, I))
    assert np.allclose(m3, want, atol=1e-15)


def test_equilibrium_at_rest_is_weights():
    assert np.array_equal(oracle.feq(1.0, np.zeros(3)), W)
    assert np.allclose(oracle.feq(0.37, np.zeros(3)), 0.37 * W, rtol=1e-15, atol=0)


# ------------------------------------------------------------------ EDM source Eq. (9)
@pytest.mark.parametrize("seed", range(5))
def test_edm_source_moments(seed):
    r = np.random.default_rng(100 + seed)
    rho = r.uniform(0.5, 1.5)
    u = r.uniform(-0.05, 0.05, 3)
    F = r.uniform(-1e-3, 1e-3, 3)
    S = oracle.edm_source(rho, u, F)
    m0, m1, m2 = moments(S)
    assert abs(m0) < 1e-15
    assert np.allclose(m1, F, rtol=0, atol=1e-15)
    up = u + F / rho
    assert np.allclose(m2, rho * (np.outer(up, up) - np.outer(u, u)), rtol=0, atol=1e-15)


# ------------------------------------------------------------------ omega_eff Eqs. (4), (7), (8)
def test_omega_eff_equal_tau():
    for tau in (0.6, 0.8, 1.0, 1.7):
        for (rr, rb) in ((1.0, 0.0), (0.3, 0.7), (0.0, 1.0)):
            assert math.isclose(oracle.omega_eff(rr, rb, tau, tau), 1.0 / tau, rel_tol=1e-14)


def test_omega_eff_pure_phases_and_mixture():
    # a pure phase relaxes at its own rate; a 50/50 mix at the harmonic-mean viscosity
    assert math.isclose(oracle.omega_eff(1.0, 0.0, 0.8, 1.4), 1 / 0.8, rel_tol=1e-14)
    assert math.isclose(oracle.omega_eff(0.0, 1.0, 0.8, 1.4), 1 / 1.4, rel_tol=1e-14)
    nu_r, nu_b = (0.8 - 0.5) / 3, (1.4 - 0.5) / 3
    nu = 1 / (0.5 / nu_r + 0.5 / nu_b)
    tau = 3 * nu + 0.5               # Eq. (4): nu = c_s^2 (tau - 1/2)
    assert math.isclose(oracle.omega_eff(0.5, 0.5, 0.8, 1.4), 1 / tau, rel_tol=1e-14)


# ------------------------------------------------------------------ BGK + EDM Eq. (1)
@pytest.mark.parametrize("seed", range(4))
def test_bgk_tau_one_gives_equilibrium_plus_source(seed):
    r = np.random.default_rng(200 + seed)
    f = W * r.uniform(0.8, 1.2, 19)
    F = r.uniform(-1e-3, 1e-3, 3)
    rho = f.sum()
    u = Cf.T @ f / rho
    out = oracle.bgk_edm(f, 1.0, F)
    want = oracle.feq(rho, u) + oracle.edm_source(rho, u, F)
    assert np.allclose(out, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("omega", [0.6, 1.0, 1.3, 1.9])
def test_bgk_moments(omega):
    f = W * rng.uniform(0.8, 1.2, 19)
    F = rng.uniform(-1e-3, 1e-3, 3)
    rho, j, P = moments(f)
    u = j / rho
    out = oracle.bgk_edm(f, omega, F)
    m0, m1, m2 = moments(out)
    assert abs(m0 - rho) < 1e-15
    assert np.allclose(m1, j + F, atol=1e-16)
    up = u + F / rho
    Peq = rho * (np.eye(3) / 3 + np.outer(u, u))
    want = (1 - omega) * P + omega * Peq + rho * (np.outer(up, up) - np.outer(u, u))
    assert np.allclose(m2, want, atol=1e-15)


# ------------------------------------------------------------------ perturbation
@pytest.mark.parametrize("seed", range(6))
def test_perturbation_moments(seed):
    r = np.random.default_rng(300 + seed)
    f = W * r.uniform(0.8, 1.2, 19)
    G = r.normal(size=3) * r.uniform(0.01, 0.5)
    omega = r.uniform(0.6, 1.8)
    sigma = r.uniform(0.005, 0.05)
    d = oracle.perturb(f, omega, sigma, G) - f
    m0, m1, m2 = moments(d)
    gm = np.linalg.norm(G)
    n = G / gm
    A = 4.5 * omega * sigma            # sigma = 2A/(9 omega)
    assert abs(m0) < 1e-15
    assert np.allclose(m1, 0, atol=1e-15)
    # capillary stress form: (A/9)|G|(n n - I); its trace-free/isotropic split fixes B_i
    assert np.allclose(m2, A / 9 * gm * (np.outer(n, n) - np.eye(3)), atol=1e-16)


def test_perturbation_skipped_at_zero_gradient():
    f = W * 1.1
    assert np.array_equal(oracle.perturb(f, 1.0, 0.02, np.array([0.0, 0.0, 5e-7])), f)


def test_perturbation_flat_interface_surface_tension():
    # A flat interface phi(x) from -1 to +1: the stress anomaly integrated across it,
    # divided by omega (steady non-equilibrium part of BGK), is sigma (I - n n) * (-1)
    # per unit |G|-integral 2 -> tangential pressure lowered by exactly sigma.
    omega, sigma = 1.0, 0.02
    f = W.copy()
    G = np.array([0.37, 0.0, 0.0])
    d = oracle.perturb(f, omega, sigma, G) - f
    P = np.einsum("ia,ib,i->ab", Cf, Cf, d) / omega
    # per unit |G|; integral of |G| across the interface is 2
    tension = -(P[1, 1] - P[0, 0]) / np.linalg.norm(G) * 2
    assert math.isclose(tension, sigma, rel_tol=1e-13)


# ------------------------------------------------------------------ recolouring
@pytest.mark.parametrize("seed", range(6))
def test_recolour_invariants(seed):
    r = np.random.default_rng(400 + seed)
    f = W * r.uniform(0.8, 1.2, 19)
    rho = f.sum()
    x = r.uniform(0, 1)
    rr, rb = x * rho, (1 - x) * rho
    G = r.normal(size=3)
    beta = 0.7
    a, b = oracle.recolour(f, rr, rb, beta, G)
    assert abs(a.sum() - rr) < 1e-15 and abs(b.sum() - rb) < 1e-15
    assert np.allclose(a + b, f, atol=1e-16)
    # colour flux: sum_i (f^r - f^b) c_i = phi j + 2 beta rho_r rho_b / rho * k n,
    # k = sum_i w_i c_ix^2/|c_i| = 2/18 + 8/(36 sqrt 2) = (1 + sqrt 2)/9
    n = G / np.linalg.norm(G)
    j = Cf.T @ f
    k = (1 + math.sqrt(2)) / 9
    want = (rr - rb) / rho * j + 2 * beta * rr * rb / rho * k * n
    assert np.allclose(Cf.T @ (a - b), want, atol=1e-16)


def test_recolour_special_cases():
    f = W * 1.05
    G = np.array([0.2, -0.1, 0.05])
    a, b = oracle.recolour(f, 0.4 * 1.05, 0.6 * 1.05, 0.0, G)   # beta = 0: proportional split
    assert np.allclose(a, 0.4 * f, rtol=1e-15) and np.allclose(b, 0.6 * f, rtol=1e-15)
    a, b = oracle.recolour(f, 1.05, 0.0, 0.7, G)                # pure red stays pure
    assert np.array_equal(b, np.zeros(19)) and np.allclose(a, f, rtol=1e-15)


# ------------------------------------------------------------------ near-contact strength
def test_A_h_shape():
    A, hmin, hcut = 0.01, 3.0, 6.0
    assert oracle.A_h(0.5, A, hmin, hcut) == A and oracle.A_h(hmin, A, hmin, hcut) == A
    assert oracle.A_h(hcut, A, hmin, hcut) == 0 and oracle.A_h(9.0, A, hmin, hcut) == 0
    assert math.isclose(oracle.A_h(hmin + 1e-9, A, hmin, hcut), A, rel_tol=1e-8)
    hs = np.linspace(hmin, hcut, 50)
    vals = np.array([oracle.A_h(h, A, hmin, hcut) for h in hs])
    assert (np.diff(vals) <= 0).all()
    # between h_min and h_cut it is an affine image of h^-3
    b3 = (hmin / hcut) ** 3
    for h in (3.5, 4.2, 5.9):
        assert math.isclose(oracle.A_h(h, A, hmin, hcut) / A * (1 - b3) + b3, (hmin / h) ** 3,
                            rel_tol=1e-13)


# ------------------------------------------------------------------ colour gradient
def _sine_field(shape, axis, k):
    nz, ny, nx = shape
    grids = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coord = {0: grids[2], 1: grids[1], 2: grids[0]}[axis]
    return np.sin(k * coord), np.cos(k * coord)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_gradient_of_sine_is_exact(axis):
    shape = (8, 10, 12)  # (nz, ny, nx)
    n = {0: 12, 1: 10, 2: 8}[axis]
    k = 2 * math.pi * 3 / n
    phi, cphi = _sine_field(shape, axis, k)
    p = oracle.make_params(12, 10, 8)
    G = oracle.gradient(p, phi)
    want = np.zeros((3,) + shape)
    want[axis] = math.sin(k) * cphi
    assert np.allclose(G, want, atol=1e-14)


def test_gradient_of_product_sine_couples_edges():
    # phi = sin(kx) sin(ly): G_x = sin k cos kx sin ly (2 + cos l)/3 (edge weights 1/36)
    shape = (4, 10, 12)
    k, l = 2 * math.pi / 12, 2 * math.pi * 2 / 10
    z, y, x = np.meshgrid(np.arange(4), np.arange(10), np.arange(12), indexing="ij")
    phi = np.sin(k * x) * np.sin(l * y)
    G = oracle.gradient(oracle.make_params(12, 10, 4), phi)
    assert np.allclose(G[0], math.sin(k) * np.cos(k * x) * np.sin(l * y) * (2 + math.cos(l)) / 3,
                       atol=1e-14)
    assert np.allclose(G[1], math.sin(l) * np.sin(k * x) * np.cos(l * y) * (2 + math.cos(k)) / 3,
                       atol=1e-14)
    assert np.allclose(G[2], 0, atol=1e-15)


def test_gradient_linear_field_and_wall_rule():
    # phi = y in a channel walled in y: exact 1 in the interior; at the walls the
    # missing neighbours take phi(x): y=0 -> 3*(1/18+4/36)*1 = 1/2, same at y=ny-1
    ny = 9
    z, y, x = np.meshgrid(np.arange(3), np.arange(ny), np.arange(4), indexing="ij")
    G = oracle.gradient(oracle.make_params(4, ny, 3, wall_y=1), y.astype(float))
    assert np.allclose(G[1][:, 1:-1, :], 1.0, atol=1e-14)
    assert np.allclose(G[1][:, 0, :], 0.5, atol=1e-15)
    assert np.allclose(G[1][:, -1, :], 0.5, atol=1e-15)
    assert np.allclose(G[0], 0, atol=1e-15) and np.allclose(G[2], 0, atol=1e-15)
