"""GPU diagnostics against the oracle's definitions: the droplet census (26-connected
components of phi > 0; integer results, compared exactly) and the radially averaged
structure factor (FP32 FFT against numpy's FP64 one; shell mode counts exactly)."""
import numpy as np
import pytest

from oracle import diagnostics
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


def _census_pair(lbm, g, periodic):
    phi = g.get_fields()["phi"]
    n, sizes = g.droplets()
    n_o, sizes_o = diagnostics.droplets(phi, periodic=periodic)
    assert n == n_o and np.array_equal(sizes, sizes_o), (n, n_o)
    return n, sizes


def test_census_of_painted_spheres_periodic_and_walled(lbm):
    shape = (24, 28, 40)
    drops = [(8.0, 8.0, 8.0, 4.0), (25.0, 9.0, 12.0, 5.0), (14.0, 20.0, 16.0, 3.5),
             (38.5, 26.0, 2.0, 3.0)]
    rr, rb = inputs.paint_droplets(shape, drops)
    nz, ny, nx = shape
    g = lbm.Lattice(lbm.make_params(nx, ny, nz))
    g.set_fields(rr, rb)
    n, _ = _census_pair(lbm, g, (True, True, True))
    assert n == 4
    g.close()
    # the same field on a lattice walled in y and z: the wrapped sphere splits
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, wall_y=1, wall_z=1))
    g.set_fields(rr, rb)
    n, _ = _census_pair(lbm, g, (True, False, False))
    assert n > 4
    g.close()


def test_census_edge_cases(lbm):
    shape = (6, 8, 10)
    nz, ny, nx = shape
    for fill in (1.0, 0.0):
        g = lbm.Lattice(lbm.make_params(nx, ny, nz))
        g.set_fields(np.full(shape, fill), np.full(shape, 1.0 - fill))
        n, sizes = g.droplets()
        assert (n, sizes.tolist()) == ((1, [nx * ny * nz]) if fill else (0, []))
        g.close()
    rr = np.zeros(shape)
    rr[1, 1, 1] = rr[2, 2, 2] = 1.0           # corner contact
    rr[4, 5, 6] = rr[4, 5, 8] = 1.0           # one node apart
    g = lbm.Lattice(lbm.make_params(nx, ny, nz))
    g.set_fields(rr, 1.0 - rr)
    n, sizes = _census_pair(lbm, g, (True, True, True))
    assert n == 3 and sizes.tolist() == [2, 1, 1]
    g.close()


def test_census_after_steps_dense_emulsion_and_channel(lbm):
    w = inputs.dense_emulsion(L=64, volume_fraction=0.3, r_range=(4.0, 7.0), seed=12)
    g = lbm.Lattice(lbm.make_params(64, 64, 64, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    g.step(40)
    # random sequential addition lets spheres touch, so the census joins them into
    # clusters; the count is whatever the definition gives, compared exactly
    n, sizes = _census_pair(lbm, g, (True, True, True))
    assert n >= 1 and sizes.sum() == int((g.get_fields()["phi"] > 0).sum())
    g.close()
    w = inputs.channel_droplets(nx=96, ny=48, nz=32, n_grid=(4, 2, 1), r_range=(5, 7), seed=9)
    nz, ny, nx = w.shape
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    g.step(30)
    n, _ = _census_pair(lbm, g, (True, False, False))
    assert n == len(w.droplets)
    g.close()


@pytest.mark.parametrize("shape", [(36, 40, 48), (32, 32, 32)])
def test_structure_factor_matches_oracle(lbm, shape):
    nz, ny, nx = shape
    w = inputs.bicontinuous(L=8, seed=3)              # parameters only
    rng = np.random.default_rng(17)
    phi0 = rng.uniform(-0.01, 0.01, size=shape)
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, **w.params))
    g.set_fields(0.5 * (1 + phi0), 0.5 * (1 - phi0))
    g.step(60)
    phi = g.get_fields()["phi"]
    nb = int(np.ceil(np.sqrt(3) * max(shape) / 2)) + 2
    k, S, m = g.structure_factor(nb)
    ko, So, mo = diagnostics.structure_factor(phi, nb)
    assert np.array_equal(m, mo)
    assert np.allclose(k, ko, rtol=1e-15, atol=0)
    assert np.abs(S - So).max() <= 1e-4 * So.max(), np.abs(S - So).max() / So.max()
    # Parseval over every mode
    assert abs((S * m).sum() - ((phi - phi.mean()) ** 2).sum()) < 1e-4 * (phi ** 2).sum()
    g.close()
