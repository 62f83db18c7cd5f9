"""Pins of the oracle's diagnostics (droplet census, structure factor) against brute
force and closed forms."""
import numpy as np

from oracle import diagnostics
from paper_2005_12764_gb300 import inputs


def _sphere(shape, c, R, periodic=(True, True, True)):
    rr, _ = inputs.paint_droplets(shape, [(c[0], c[1], c[2], R)], periodic=periodic)
    return rr > 0.5


def test_census_of_separated_spheres_is_their_painted_volumes():
    shape = (24, 28, 40)
    drops = [(8.0, 8.0, 8.0, 4.0), (25.0, 9.0, 12.0, 5.0), (14.0, 20.0, 16.0, 3.5),
             (38.5, 26.0, 2.0, 3.0)]                 # the last one wraps in x, y and z
    masks = [_sphere(shape, d[:3], d[3]) for d in drops]
    phi = np.where(np.any(masks, axis=0), 1.0, -1.0)
    n, sizes = diagnostics.droplets(phi)
    assert n == len(drops)
    assert sizes.tolist() == sorted((int(m.sum()) for m in masks), reverse=True)


def test_census_connectivity_and_walls():
    shape = (6, 8, 10)
    phi = -np.ones(shape)
    phi[1, 1, 1] = phi[2, 2, 2] = 1.0               # corner contact: one component
    phi[4, 5, 6] = phi[4, 5, 8] = 1.0               # one empty node between: two
    n, sizes = diagnostics.droplets(phi)
    assert n == 3 and sizes.tolist() == [2, 1, 1]
    slab = -np.ones(shape)
    slab[:, 0, :] = slab[:, -1, :] = 1.0            # rows y = 0 and y = ny - 1
    assert diagnostics.droplets(slab)[0] == 1
    assert diagnostics.droplets(slab, periodic=(True, False, True))[0] == 2
    n, sizes = diagnostics.droplets(np.ones(shape))
    assert n == 1 and sizes.tolist() == [int(np.prod(shape))]
    assert diagnostics.droplets(-np.ones(shape))[0] == 0


def test_structure_factor_of_one_mode_and_parseval():
    L, m0 = 16, 3
    x = np.arange(L)
    phi = np.broadcast_to(np.cos(2 * np.pi * m0 * x / L), (L, L, L)).copy()
    k, S, cnt = diagnostics.structure_factor(phi, 20)
    N = L ** 3
    # |phi_hat|^2 = (N/2)^2 at m = +-m0 e_x: all of it in shell m0
    assert abs(S[m0] - N / (2 * cnt[m0])) < 1e-9 * N
    assert np.abs(np.delete(S, m0)).max() < 1e-18 * N
    # Parseval: every mode of a 16^3 box lies in shells < 20 (|m| <= sqrt(3) 8)
    r = np.random.default_rng(2).normal(size=(L, L, L))
    k, S, cnt = diagnostics.structure_factor(r, 20)
    assert abs((S * cnt).sum() - ((r - r.mean()) ** 2).sum()) < 1e-9 * r.size
    assert abs(k[1] - 2 * np.pi / L) < 1e-15
