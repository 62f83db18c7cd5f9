"""Seeded synthetic inputs for the colour-gradient LB workloads.

This module draws random numbers and paints initial density fields; it holds none
of the lattice Boltzmann arithmetic, so both the FP64 oracle (in tests) and the GPU
library are fed from it. The paper uses no public dataset: its microfluidic-crystal,
dense-emulsion and bicontinuous-gel runs (Secs. "LB method for microfluidic
crystals" and "High-performance LB code for bijel materials") are stood in for by
the generators below, all driven by NumPy PCG64 ``default_rng(seed)``.

Arrays are float64 and indexed [z, y, x] (x fastest in memory). Red is the
dispersed phase: rho_r = 1 inside a droplet, rho_b = 1 outside, sharp interface,
and a node is inside when |x - c|^2 < R^2 (strict, minimum image along periodic
axes).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    """Initial fields plus the physical parameters of one synthetic run."""
    name: str
    shape: tuple            # (nz, ny, nx)
    rho_r: np.ndarray
    rho_b: np.ndarray
    params: dict            # keyword parameters of the lattice (tau, sigma, ...)
    droplets: list = dataclasses.field(default_factory=list)   # [(cx, cy, cz, R)]
    pins: np.ndarray | None = None
    steps: int = 0


def paint_droplets(shape, droplets, periodic=(True, True, True)):
    """rho_r, rho_b for red spheres [(cx, cy, cz, R), ...] in blue fluid.

    periodic = (x, y, z) flags; spheres wrap across periodic axes only.
    """
    nz, ny, nx = shape
    red = np.zeros(shape, dtype=bool)
    n3 = (nx, ny, nz)
    for (cx, cy, cz, R) in droplets:
        c = (cx, cy, cz)
        ranges = []
        for a in range(3):
            lo = int(math.floor(c[a] - R)) - 1
            hi = int(math.ceil(c[a] + R)) + 1
            idx = np.arange(lo, hi + 1)
            d = idx - c[a]
            if periodic[a]:
                idx = np.mod(idx, n3[a])
            else:
                keep = (idx >= 0) & (idx < n3[a])
                idx, d = idx[keep], d[keep]
            ranges.append((idx, d))
        (ix, dx), (iy, dy), (iz, dz) = ranges
        r2 = dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dx[None, None, :] ** 2
        inside = r2 < R * R
        sub = red[np.ix_(iz, iy, ix)]
        red[np.ix_(iz, iy, ix)] = sub | inside
    rho_r = red.astype(np.float64)
    rho_b = 1.0 - rho_r
    return rho_r, rho_b


def static_droplet(L=32, R=8.0, sigma=0.01, tau=1.0, beta=0.7, steps=500):
    """Static droplet: one red sphere of radius R at the centre of a periodic L^3 box."""
    c = L / 2.0
    rr, rb = paint_droplets((L, L, L), [(c, c, c, R)])
    return Workload(f"static-droplet-{L}^3-R{R:g}", (L, L, L), rr, rb,
                    dict(tau_r=tau, sigma=sigma, beta=beta, A_nc=0.0), [(c, c, c, R)],
                    steps=steps)


def _min_image(d, n):
    return d - n * np.round(d / n)


def channel_droplets(nx=256, ny=128, nz=64, n_grid=(10, 2, 2), r_range=(6.0, 9.0), gap=2.0,
                     wall_clear=2.0, seed=1002, sigma=0.02, tau=1.0, beta=0.7, A_nc=0.01,
                     h_min=3.0, g_x=1e-6, steps=10_000, max_tries=100_000):
    """Microfluidic-crystal channel: droplets on a jittered n_grid lattice.

    Walls (halfway bounce-back) at the y and z extremes, periodic in x. Radii are
    uniform in r_range; each droplet is placed by rejection inside its lattice cell
    so that surfaces stay >= gap apart (x periodic) and >= wall_clear from the
    walls (walls at -1/2 and n - 1/2).
    """
    rng = np.random.default_rng(seed)
    gx, gy, gz = n_grid
    cells = [(i, j, k) for k in range(gz) for j in range(gy) for i in range(gx)]
    drops = []
    for (i, j, k) in cells:
        R = float(rng.uniform(*r_range))
        lo = np.array([i * nx / gx, j * ny / gy, k * nz / gz])
        hi = lo + np.array([nx / gx, ny / gy, nz / gz])
        for _ in range(max_tries):
            c = rng.uniform(lo, hi)
            if c[1] - R < -0.5 + wall_clear or c[1] + R > ny - 0.5 - wall_clear:
                continue
            if c[2] - R < -0.5 + wall_clear or c[2] + R > nz - 0.5 - wall_clear:
                continue
            ok = True
            for (dx_, dy_, dz_, R2) in drops:
                d = np.array([_min_image(c[0] - dx_, nx), c[1] - dy_, c[2] - dz_])
                if np.sqrt((d * d).sum()) < R + R2 + gap:
                    ok = False
                    break
            if ok:
                drops.append((float(c[0]), float(c[1]), float(c[2]), R))
                break
        else:
            raise RuntimeError("could not place droplet")
    rr, rb = paint_droplets((nz, ny, nx), drops, periodic=(True, False, False))
    params = dict(wall_y=1, wall_z=1, tau_r=tau, sigma=sigma, beta=beta, A_nc=A_nc,
                  h_min=h_min, g=(g_x, 0.0, 0.0))
    return Workload(f"channel-{nx}x{ny}x{nz}-{len(drops)}drops", (nz, ny, nx), rr, rb, params,
                    drops, steps=steps)


def channel_shan_chen(G_sc=1.6, fill=0.02, **kw):
    """The microfluidic-crystal channel (same droplets, walls and body force) for the
    Shan-Chen model: each species 0.96 of its colour-model density plus `fill`
    everywhere (a separated Shan-Chen mixture keeps a little of each species in both
    phases), coupling G_sc, no near-contact force (it belongs to the colour model)."""
    w = channel_droplets(**kw)
    params = dict(wall_y=1, wall_z=1, tau_r=w.params["tau_r"], g=w.params["g"],
                  model="shan_chen", G_sc=G_sc)
    scale = 1.0 - 2.0 * fill
    return Workload(w.name.replace("channel", "channel-shan-chen"), w.shape,
                    scale * w.rho_r + fill, scale * w.rho_b + fill, params, w.droplets,
                    steps=w.steps)


def dense_emulsion(L=512, volume_fraction=0.35, r_range=(6.0, 12.0), seed=1003, sigma=0.01,
                   tau=1.0, beta=0.7, A_nc=0.01, h_min=3.0, kolmogorov_amp=1e-5,
                   max_attempts=10_000_000, steps=2000):
    """Dense emulsion: random non-overlapping spheres (random sequential addition).

    Radii are drawn uniform in r_range, sorted largest first, and each is placed at
    uniformly random centres until it overlaps no earlier sphere (cell list,
    periodic); stops when the target volume fraction is reached or the attempt
    budget is spent (the achieved fraction is returned in params).
    """
    rng = np.random.default_rng(seed)
    target = volume_fraction * L ** 3
    radii = []
    vol = 0.0
    while vol < target:
        r = float(rng.uniform(*r_range))
        radii.append(r)
        vol += 4.0 / 3.0 * math.pi * r ** 3
    radii.sort(reverse=True)
    rmax = r_range[1]
    cell = 2 * rmax
    nc = max(1, int(L // cell))
    csz = L / nc
    grid = {}
    drops = []
    attempts = 0
    placed_vol = 0.0
    for r in radii:
        placed = False
        while attempts < max_attempts:
            attempts += 1
            c = rng.uniform(0, L, size=3)
            ci = (c // csz).astype(int) % nc
            ok = True
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        key = ((ci[0] + dx) % nc, (ci[1] + dy) % nc, (ci[2] + dz) % nc)
                        for k in grid.get(key, ()):
                            o = drops[k]
                            d = _min_image(c - np.array(o[:3]), L)
                            if (d * d).sum() < (r + o[3]) ** 2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                drops.append((float(c[0]), float(c[1]), float(c[2]), r))
                grid.setdefault(tuple(ci), []).append(len(drops) - 1)
                placed_vol += 4.0 / 3.0 * math.pi * r ** 3
                placed = True
                break
        if not placed:
            break
    rr, rb = paint_droplets((L, L, L), drops)
    params = dict(tau_r=tau, sigma=sigma, beta=beta, A_nc=A_nc, h_min=h_min,
                  kolmogorov_amp=kolmogorov_amp)
    w = Workload(f"emulsion-{L}^3", (L, L, L), rr, rb, params, drops, steps=steps)
    w.params_extra = {"achieved_fraction": placed_vol / L ** 3, "attempts": attempts}
    return w


def bicontinuous(L=640, amplitude=0.01, pin_fraction=0.02, seed=1005, sigma=0.015, tau=0.8,
                 beta=0.7, A_nc=0.02, h_min=3.0, steps=20_000):
    """Bicontinuous gel quench: symmetric mixture with uniform colour noise.

    phi0 ~ U(-amplitude, amplitude); rho_r = (1 + phi0)/2, rho_b = (1 - phi0)/2;
    a fraction pin_fraction of nodes, drawn without replacement, are pinning sites.
    """
    rng = np.random.default_rng(seed)
    shape = (L, L, L)
    phi0 = rng.uniform(-amplitude, amplitude, size=shape)
    rr = 0.5 * (1.0 + phi0)
    rb = 0.5 * (1.0 - phi0)
    N = L ** 3
    npin = int(round(pin_fraction * N))
    pins = np.zeros(N, dtype=np.uint8)
    pins[rng.choice(N, size=npin, replace=False)] = 1
    params = dict(tau_r=tau, sigma=sigma, beta=beta, A_nc=A_nc, h_min=h_min)
    return Workload(f"bicontinuous-{L}^3", shape, rr, rb, params, [], pins.reshape(shape),
                    steps=steps)


def sheared_bijel(nx=1024, ny=128, nz=128, amplitude=0.01, wall_u=0.01, seed=1006,
                  sigma=0.015, tau=0.8, beta=0.7, A_nc=0.02, h_min=3.0, steps=500_000):
    """Confined bicontinuous mixture under shear (the sheared-bijel channel of the
    paper's bijel section, 128 x 128 x 1024 with a periodic mainstream axis).

    Layout here: x is the periodic mainstream axis (nx = 1024); the walls at the y
    extremes slide with +-wall_u along x (shear 2 wall_u / ny); the walls at the z
    extremes are at rest. Symmetric mixture with uniform colour noise,
    phi0 ~ U(-amplitude, amplitude). The paper's colloids are not modelled; the
    near-contact force stands in for what arrests the coarsening.
    """
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    phi0 = rng.uniform(-amplitude, amplitude, size=shape)
    rr = 0.5 * (1.0 + phi0)
    rb = 0.5 * (1.0 - phi0)
    params = dict(wall_y=1, wall_z=1, wall_u=wall_u, tau_r=tau, sigma=sigma, beta=beta,
                  A_nc=A_nc, h_min=h_min)
    return Workload(f"sheared-bijel-{nx}x{ny}x{nz}", shape, rr, rb, params, [], steps=steps)


def random_state(shape, seed, amp=0.05, u_amp=0.02):
    """Smooth-ish random two-phase fields for unit tests: rho_k in (0.2, 1.2)-ish."""
    rng = np.random.default_rng(seed)
    phi = np.tanh(3.0 * rng.uniform(-1, 1, size=shape))
    rho = 1.0 + amp * rng.uniform(-1, 1, size=shape)
    rr = 0.5 * rho * (1 + phi)
    rb = 0.5 * rho * (1 - phi)
    u = u_amp * rng.uniform(-1, 1, size=(3,) + tuple(shape))
    return rr, rb, u


def serving_requests(n=256, seed=1004, rate_hz=50.0, edges=(32, 48, 64, 96, 128),
                     sigma_range=(0.005, 0.03), steps_range=(200, 2000)):
    """Seeded request stream: box edge, droplet radius L/4, sigma, steps, arrival time.

    Half the requests (drawn at random) are static droplets, half are sheared by a
    Kolmogorov force 1e-5 sin(2 pi y / L). Arrivals are a Poisson process.
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for k in range(n):
        L = int(rng.choice(edges))
        reqs.append(dict(id=k, arrival_s=float(t[k]), L=L, R=L / 4.0,
                         sigma=float(rng.uniform(*sigma_range)),
                         steps=int(rng.integers(steps_range[0], steps_range[1] + 1)),
                         sheared=bool(rng.integers(0, 2))))
    return reqs
