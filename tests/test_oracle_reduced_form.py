"""Pins of the reduced (Q + 5) storage form on the FP64 oracle.

After recolouring, a node's two species hold
    f^r_i = kappa_r f_i + w_i (c_i . m) / |c_i|,   f^b_i = kappa_b f_i - w_i (c_i . m) / |c_i|,
with f_i = f^r_i + f^b_i, kappa_k = rho_k / rho and m = beta (rho_r rho_b / rho) n, n the
unit colour gradient of the step (m = 0 where the gradient vanishes). The GPU
library's reduced storage keeps only f_i and (kappa_r, kappa_b, m) per node and
rebuilds the species from them, so the form must hold exactly for every state the
method produces. These tests check it on oracle states: the red excess
f^r_i - kappa_r f_i must lie in the 3-dimensional span of w_i c_i / |c_i| (19 numbers
per node, a strong constraint), and m must have the length beta rho_r rho_b / rho and
the direction of the colour gradient. The projection constant used to recover m,
sum_i (w_i / |c_i|) c_i c_i = (1 + sqrt 2)/9 I, is checked by brute force.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2005_12764_gb300 import inputs

C, W, OPP, B = oracle.lattice()
Cf = C.astype(float)
CLEN = np.sqrt((Cf * Cf).sum(1))
WC = np.where(CLEN > 0, W / np.where(CLEN > 0, CLEN, 1.0), 0.0)   # w_i / |c_i|, 0 at rest


def test_projection_constant_brute_force():
    M = np.zeros((3, 3))
    for i in range(19):
        M += WC[i] * np.outer(Cf[i], Cf[i])
    assert np.allclose(M, np.eye(3) * (1 + math.sqrt(2)) / 9, rtol=0, atol=1e-15)


def split(fr, fb):
    """(total, kappa_r, kappa_b, m, share) of the species populations [19, ...]."""
    t = fr + fb
    rr, rb = fr.sum(0), fb.sum(0)
    kr, kb = rr / (rr + rb), rb / (rr + rb)
    d = fr - kr * t
    m = np.einsum("ia,i...->a...", Cf, d) * (9.0 / (1.0 + math.sqrt(2.0)))
    share = np.einsum("i,ia,a...->i...", WC, Cf, m)
    return t, kr, kb, m, share


CASES = {
    # walls in y and z sliding in x, near contact, body force, unequal viscosities
    "walls_sliding_nc_var_tau": dict(
        shape=(12, 22, 30), periodic=(True, False, False),
        drops=[(9.0, 8.0, 6.0, 4.5), (19.5, 12.0, 6.0, 4.5)],
        kw=dict(wall_y=1, wall_z=1, wall_u=0.02, tau_r=0.8, tau_b=1.1, sigma=0.02, beta=0.7,
                A_nc=0.02, h_min=3.0, g=(1e-5, 0, 0))),
    # periodic box, Kolmogorov forcing, weak segregation
    "periodic_kolmogorov": dict(
        shape=(16, 16, 16), periodic=(True, True, True),
        drops=[(8.0, 8.0, 8.0, 5.0)],
        kw=dict(sigma=0.01, beta=0.3, kolmogorov_amp=1e-4)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_recoloured_states_have_the_reduced_form(case):
    c = CASES[case]
    nz, ny, nx = c["shape"]
    rr, rb = inputs.paint_droplets(c["shape"], c["drops"], periodic=c["periodic"])
    P = oracle.make_params(nx, ny, nz, **c["kw"])
    o = oracle.Lattice(P)
    o.set_fields(rr, rb)
    o.step(7)
    fr, fb = o.get_pops()
    f = o.get_fields()
    o.close()
    t, kr, kb, m, share = split(fr, fb)
    # the excess lies in the span of w_i c_i / |c_i| for both species, opposite signs
    assert np.abs(fr - (kr * t + share)).max() <= 1e-14
    assert np.abs(fb - (kb * t - share)).max() <= 1e-14
    # |m| = beta rho_r rho_b / rho and m along the colour gradient where the gradient
    # is well above the threshold below which the recolouring angle is undefined;
    # m = 0 well below it
    G = oracle.gradient(P, f["phi"])
    gm = np.sqrt((G * G).sum(0))
    beta = c["kw"]["beta"]
    want = beta * f["rho_r"] * f["rho_b"] / (f["rho_r"] + f["rho_b"])
    mm = np.sqrt((m * m).sum(0))
    big = gm >= 1e-5
    assert big.sum() > 100
    assert np.abs(mm[big] - want[big]).max() <= 1e-12 * max(1.0, want.max())
    cos = (m * G).sum(0)[big] / (mm[big] * gm[big])
    assert np.abs(cos - 1.0).max() <= 1e-9
    small = gm < 1e-7
    if small.any():
        assert mm[small].max() <= 1e-15


def test_a_wrong_recolouring_weight_breaks_the_form():
    # the same check on a split whose recolouring term lacks the 1/|c_i| factor: the
    # excess then leaves the span, so the check above would catch such a mistake
    rng = np.random.default_rng(3)
    t = np.abs(rng.normal(0.05, 0.01, size=(19, 50)))
    kr = rng.uniform(0.1, 0.9, size=50)
    m = rng.normal(size=(3, 50)) * 0.01
    wrong = np.einsum("i,ia,a...->i...", W * (CLEN > 0), Cf, m)
    fr = kr * t + wrong
    fb = (1 - kr) * t - wrong
    _, kr2, _, _, share = split(fr, fb)
    assert np.abs(fr - (kr2 * t + share)).max() > 1e-6
