"""Full-size workloads on the GPU, in the launch configuration of the benchmark.

- Dense emulsion: 512^3 periodic, random non-overlapping droplets (volume fraction
  0.35, radii uniform in [6, 12]), Kolmogorov forcing 1e-5 sin(2 pi y / 512),
  near-contact force on.
- Bicontinuous gel quench: 640^3 periodic, symmetric mixture with colour noise of
  amplitude 0.01 and 2 % pinning sites, tau = 0.8, sigma = 0.015, A_nc = 0.02.
- Sheared bijel channel: 1024 x 128 x 128, walls at the y extremes sliding with
  +-0.01 along the periodic x axis, walls at the z extremes at rest, symmetric
  mixture with colour noise 0.01 (samples away from the walls, so that the
  periodic window holds everything the centre depends on).

The oracle cannot hold these lattices, so each is checked in two ways:
1. at sampled nodes, one step at a time: a cube of 2R+1 nodes around each sample
   (R = 12 covers the pull, the gradient of the pulled densities and the
   near-contact rays of the lagged field, at most h_cut + 3 = 9 nodes) is copied
   out of the GPU state, the oracle steps that cube as a periodic lattice of its
   own, and the GPU's next-step populations at the sample must match the oracle's
   at the cube's centre (nodes further out are wrong in the oracle's cube, but the
   centre depends on none of them);
2. by invariants that hold at any size: each species' mass is conserved and every
   value stays finite.
"""
import math

import numpy as np
import pytest

import branch_cases
import oracle
from paper_2005_12764_gb300 import inputs

pytestmark = pytest.mark.gpu

R = 12
W = 2 * R + 1


@pytest.fixture(scope="module")
def lbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12764_gb300 import build_lib, lbm as L
    build_lib.build()
    L.load()
    return L


def _map_to_oracle(lbm):
    """index map: oracle direction k -> library direction."""
    cg = lbm.velocity_set()
    co = oracle.lattice()[0]
    return np.array([int(np.nonzero((cg == co[k]).all(1))[0][0]) for k in range(19)])


def _window_params(params, shape, y_centre):
    """Oracle parameters of a window cube: Kolmogorov forcing depends on the
    absolute row, so it enters as the uniform force the centre row feels. Windows
    are periodic: on walled lattices they are taken away from the walls, where
    nothing the centre depends on reaches the window's edge."""
    kw = dict(params)
    for k in ("wall_y", "wall_z", "wall_u"):
        kw.pop(k, None)
    ny = shape[1]
    amp = kw.pop("kolmogorov_amp", 0.0)
    g = list(kw.pop("g", (0.0, 0.0, 0.0)))
    g[0] += amp * math.sin(2.0 * math.pi * y_centre / ny)
    return oracle.make_params(W, W, W, g=tuple(g), **kw)


def _check_sampled_step(lbm, g, w, samples, pins=None):
    """(worst difference, samples whose difference is not a threshold branch, samples
    that are): a sample whose next-step populations differ from the oracle's by more
    than 1e-6 passes only if the GPU's A_h there is the oracle's with a threshold of
    the film measurement moved by its FP32 rounding bound, and the oracle's step with
    that A_h gives the GPU's populations."""
    m = _map_to_oracle(lbm)
    nz, ny, nx = w.shape
    before = [g.get_window(x - R, y - R, z - R, W, W, W) for (x, y, z) in samples]
    ah_gpu = g.get_nc_field() if w.params.get("A_nc", 0.0) > 0 else None
    g.step(1)
    worst, bad, branches = 0.0, 0, 0
    for (x, y, z), (fr, fb, lag) in zip(samples, before):
        P = _window_params(w.params, w.shape, y)
        pw = None
        if pins is not None:
            zz = (np.arange(z - R, z + R + 1) % nz)[:, None, None]
            yy = (np.arange(y - R, y + R + 1) % ny)[None, :, None]
            xx = (np.arange(x - R, x + R + 1) % nx)[None, None, :]
            pw = pins[zz, yy, xx].ravel()
        centre = (R * W + R) * W + R
        oa, ob, _ = oracle.step_nodes(P, fr.reshape(19, -1)[m], fb.reshape(19, -1)[m],
                                      lag.ravel(), np.array([centre]), pin=pw)
        gr, gb, _ = g.get_window(x, y, z, 1, 1, 1)
        d = max(np.abs(oa[0] - gr.reshape(19)[m]).max(), np.abs(ob[0] - gb.reshape(19)[m]).max())
        worst = max(worst, d)
        if d > 1e-6:
            if ah_gpu is not None and branch_cases.step_explained(
                    P, fr.reshape(19, -1)[m], fb.reshape(19, -1)[m], lag.ravel(), centre,
                    gr.reshape(19)[m], gb.reshape(19)[m], float(ah_gpu[z, y, x]), pin=pw):
                branches += 1
            else:
                bad += 1
    return worst, bad, branches


def _samples(rng, shape, droplets, n_any, n_iface):
    """n_any uniformly random nodes, plus n_iface nodes on droplet surfaces (the
    nearest node to a random point of a random droplet's sphere)."""
    nz, ny, nx = shape
    out = [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz)))
           for _ in range(n_any)]
    for _ in range(n_iface if droplets else 0):
        cx, cy, cz, r = droplets[int(rng.integers(len(droplets)))]
        d = rng.normal(size=3)
        p = np.array([cx, cy, cz]) + r * d / np.linalg.norm(d)
        out.append((int(round(p[0])) % nx, int(round(p[1])) % ny, int(round(p[2])) % nz))
    return out


_EMULSION = {}


def _emulsion():
    if "w" not in _EMULSION:
        _EMULSION["w"] = inputs.dense_emulsion()   # 512^3, volume fraction 0.35, radii 6-12
    return _EMULSION["w"]


@pytest.mark.parametrize("storage", ["fp32", "fp32_q5"])
def test_dense_emulsion_512_full_size(lbm, storage):
    # the full FP32 form and the reduced (Q + 5) form, the latter holding 25.8 GB for
    # the two copies instead of 40.8 GB
    w = _emulsion()
    assert w.params_extra["achieved_fraction"] > 0.34
    n = w.shape[0]
    g = lbm.Lattice(lbm.make_params(n, n, n, storage=storage, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    m0 = g.observables()
    g.step(20)
    samples = _samples(np.random.default_rng(31), w.shape, w.droplets, 6, 10)
    worst, bad, branches = _check_sampled_step(lbm, g, w, samples)
    print(f"emulsion 512^3 ({storage}): worst |d f| at samples", worst, "branches", branches)
    assert bad == 0, worst
    m1 = g.observables()
    assert np.isfinite(m1[:5]).all()
    # per-species mass: FP32 arithmetic on 1.3e8 nodes, relative drift well below 1e-6
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-6 and abs(m1[1] - m0[1]) / m0[1] < 1e-6
    # droplet census: random sequential addition lets spheres touch (near the jamming
    # fraction they form clusters), so it reports clusters; the components cover
    # exactly the positive nodes
    n, sizes = g.droplets()
    phi = g.get_fields()["phi"]
    print("emulsion 512^3: components", n, "of", len(w.droplets), "placed; largest", sizes[:3])
    assert 1 <= n <= len(w.droplets)
    assert sizes.sum() == int((phi > 0).sum())
    g.close()


def test_bicontinuous_gel_640_full_size(lbm):
    w = inputs.bicontinuous()          # 640^3, noise 0.01, 2 % pins
    n = w.shape[0]
    g = lbm.Lattice(lbm.make_params(n, n, n, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    g.set_pin_mask(w.pins)
    m0 = g.observables()
    g.step(10)
    # every node of the noise field lies on an interface
    samples = _samples(np.random.default_rng(32), w.shape, [], 16, 0)
    worst, bad, branches = _check_sampled_step(lbm, g, w, samples, pins=w.pins)
    print("gel 640^3: worst |d f| at samples", worst, "branches", branches)
    # a film measurement with a sample within FP32 rounding of a threshold may take
    # the other branch in FP32; every other difference fails
    assert bad == 0, worst
    m1 = g.observables()
    assert np.isfinite(m1[:5]).all()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-6 and abs(m1[1] - m0[1]) / m0[1] < 1e-6
    # structure factor: every mode is in a shell below 560 (|m| <= sqrt(3) 320), so
    # the shells sum to the variance of phi (Parseval)
    k, S, modes = g.structure_factor(560)
    phi = g.get_fields()["phi"]
    var = ((phi - phi.mean()) ** 2).sum()
    assert modes.sum() == phi.size
    assert abs((S * modes).sum() - var) < 1e-3 * var
    print("gel 640^3: S(k) peak at k =", k[1 + int(np.argmax(S[1:]))])
    g.close()


def test_sheared_bijel_channel_full_size(lbm):
    w = inputs.sheared_bijel()         # 1024 x 128 x 128, sliding y-walls
    nz, ny, nx = w.shape
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    m0 = g.observables()
    g.step(20)
    rng = np.random.default_rng(33)
    samples = [(int(rng.integers(nx)), int(rng.integers(R, ny - R)), int(rng.integers(R, nz - R)))
               for _ in range(16)]
    worst, bad, branches = _check_sampled_step(lbm, g, w, samples)
    print("sheared bijel: worst |d f| at samples", worst, "branches", branches)
    assert bad == 0, worst
    m1 = g.observables()
    assert np.isfinite(m1[:5]).all()
    assert abs(m1[0] - m0[0]) / m0[0] < 1e-6 and abs(m1[1] - m0[1]) / m0[1] < 1e-6
    # the walls drag the fluid: x momentum near the top wall is positive, near the
    # bottom wall negative
    f = g.get_fields()
    ux = f["u"][0].mean(axis=(0, 2))
    assert ux[-1] > 0 > ux[0]
    g.close()
