"""Pins of the oracle's Shan-Chen binary mixture (Sec. "Multi-component flows",
Eqs. (5)-(9) and (12)): the cohesive force against its closed form on a sine
profile, Newton's third law for the total force, conservation of species mass and
of momentum, the spinodal threshold G rho = 2 (tau - 1/2)/tau of the symmetric
mixture (either side of it, a composition perturbation grows or decays), the reduction to the
single-fluid colour-gradient step when one species is absent, and the independent
numpy mini-oracle.
"""
import numpy as np
import pytest

import oracle
from oracle import mini
from paper_2005_12764_gb300 import inputs

C, W, OPP, B = oracle.lattice()


def _lat(shape, **kw):
    nz, ny, nx = shape
    return oracle.Lattice(oracle.make_params(nx, ny, nz, model="shan_chen", **kw))


def _pre_stream(rho):
    """Populations whose pull-streaming gives densities exactly rho: f_i(x) =
    w_i rho(x + c_i), so that f_i(x - c_i) = w_i rho(x)."""
    f = np.empty((19,) + rho.shape)
    for i in range(19):
        f[i] = W[i] * np.roll(rho, shift=(-C[i][2], -C[i][1], -C[i][0]), axis=(0, 1, 2))
    return f


def test_cohesive_force_matches_closed_form_on_a_sine():
    # rho_b = 1 + eps sin(k x), rho_r = 1 after streaming: sum_i w_i rho_b(x + c_i) c_ix
    # = eps cos(k x) sin(k) / 3, so F_x = -G eps cos(k x) sin(k) / 3 (F^b = 0)
    nx, eps, G = 16, 0.01, 1.3
    shape = (3, 3, nx)
    k = 2 * np.pi / nx
    x = np.arange(nx)
    rb = np.broadcast_to(1 + eps * np.sin(k * x), shape).copy()
    rr = np.ones(shape)
    lat = _lat(shape, G_sc=G)
    lat.set_pops(_pre_stream(rr), _pre_stream(rb), (rr - rb) / (rr + rb))
    lat.step(1)
    F = lat.get_forces()
    want = -G * eps * np.cos(k * x) * np.sin(k) / 3
    assert np.abs(F[0] - want[None, None, :]).max() < 1e-15
    assert np.abs(F[1]).max() < 1e-16 and np.abs(F[2]).max() < 1e-16


def test_total_cohesive_force_vanishes_and_momentum_is_conserved():
    shape = (6, 5, 7)
    rr, rb, u = inputs.random_state(shape, seed=21)
    lat = _lat(shape, G_sc=2.2, tau_r=0.9)
    lat.set_fields(rr, rb, u)
    m0 = lat.totals()
    for _ in range(5):
        lat.step(1)
        F = lat.get_forces()
        assert np.abs(F.reshape(3, -1).sum(1)).max() < 1e-13
    m1 = lat.totals()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-13 and abs(m1[1] - m0[1]) / m0[1] < 1e-13
    assert np.abs(np.array(m1[2:5]) - np.array(m0[2:5])).max() < 1e-13


@pytest.mark.parametrize("tau", [1.0, 0.8])
@pytest.mark.parametrize("ratio, grows", [(0.85, False), (1.25, True)])
def test_spinodal_threshold_of_the_symmetric_mixture(tau, ratio, grows):
    # rho_r = rho_b = 1/2 (rho = 1) with a long-wave composition perturbation. The
    # mean-field free energy c_s^2 [sum_k rho_k ln rho_k + G rho_r rho_b] turns
    # concave at G rho = 2; in this lattice model the composition diffuses with
    # c_s^2 (tau - 1/2) while the cohesive force drives it with mobility tau (each
    # species' velocity is reset to the common u plus F^k/rho_k every step), so the
    # threshold is G rho = 2 (tau - 1/2)/tau. Below it the perturbation decays,
    # above it grows; a sign error or a factor 2 in the force flips a case.
    nx = 32
    shape = (2, 2, nx)
    x = np.arange(nx)
    d = 1e-3 * np.sin(2 * np.pi * x / nx)
    rr = np.broadcast_to(0.5 + d, shape).copy()
    rb = np.broadcast_to(0.5 - d, shape).copy()
    G = ratio * 2 * (tau - 0.5) / tau
    lat = _lat(shape, G_sc=G, tau_r=tau)
    lat.set_fields(rr, rb)
    lat.step(800)
    f = lat.get_fields()
    amp = np.abs(f["rho_r"] - f["rho_b"]).max() / 2
    assert (amp > 1.5e-3) if grows else (amp < 0.9e-3), amp


def test_one_species_reduces_to_the_single_fluid_step():
    # no blue fluid: the Shan-Chen step is the BGK + EDM step of the red fluid, the
    # same as the colour-gradient step (whose recolouring then gives all to red)
    ny, g = 16, 1e-5
    shape = (2, ny, 3)
    rr, _, u = inputs.random_state(shape, seed=4)
    rb = np.zeros(shape)
    kw = dict(wall_y=1, tau_r=0.8, g=(g, 0, 0))
    a = _lat(shape, G_sc=1.7, **kw)
    nz, ny_, nx = shape
    b = oracle.Lattice(oracle.make_params(nx, ny_, nz, sigma=0.0, beta=0.0, **kw))
    for lat in (a, b):
        lat.set_fields(rr, rb, u)
        lat.step(20)
    fa, fb = a.get_pops(), b.get_pops()
    assert np.abs(fa[0] - fb[0]).max() < 1e-15 and not fa[1].any()


@pytest.mark.parametrize("case", [
    dict(shape=(5, 6, 7), G_sc=1.8),
    dict(shape=(6, 7, 5), G_sc=2.4, wall_y=1, wall_z=1, tau_b=0.8, g=(1e-4, 0, 2e-5)),
])
def test_numpy_mini_oracle_agrees(case):
    case = dict(case)
    shape = case.pop("shape")
    nz, ny, nx = shape
    rr, rb, u = inputs.random_state(shape, seed=sum(shape) + 7)
    lat = _lat(shape, **case)
    lat.set_fields(rr, rb, u)
    m = mini.MiniLattice(nx, ny, nz, model="shan_chen", **case)
    m.set_fields(rr, rb, u)
    lat.step(4)
    m.step(4)
    f = lat.get_fields()
    for k in ("rho_r", "rho_b", "phi"):
        assert np.allclose(f[k], m.last[k], rtol=0, atol=1e-13), k
    assert np.allclose(f["u"], m.last["u"], rtol=0, atol=1e-13)
    assert np.allclose(lat.get_forces(), m.last["F"], rtol=0, atol=1e-13)


def test_step_nodes_matches_full_step():
    shape = (8, 9, 10)
    rr, rb, u = inputs.random_state(shape, seed=8)
    kw = dict(G_sc=2.0, wall_y=1, g=(1e-4, 0, 0))
    lat = _lat(shape, **kw)
    lat.set_fields(rr, rb, u)
    lat.step(2)
    fr, fb = lat.get_pops()
    lag = lat.get_phi_lag()
    nodes = np.random.default_rng(3).choice(fr[0].size, 200, replace=False)
    lat.step(1)
    gr, gb = lat.get_pops()
    p = oracle.make_params(shape[2], shape[1], shape[0], model="shan_chen", **kw)
    oa, ob, F = oracle.step_nodes(p, fr.reshape(19, -1), fb.reshape(19, -1), lag.ravel(), nodes)
    assert np.array_equal(oa, gr.reshape(19, -1)[:, nodes].T)
    assert np.array_equal(ob, gb.reshape(19, -1)[:, nodes].T)
