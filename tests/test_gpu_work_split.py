"""GPU checks of how the step's work is split and bounded.

- Chain mode of the step kernel (lattices of fewer tiles than the GPU holds CTAs:
  bands of planes one CTA per (band, tile), the planes above shared in runs that may
  end inside one tile and continue on the next) against the FP64 oracle, and bitwise
  against part mode (the serving engine's split) on the same lattice.
- The near-contact pass (blocks of nodes with halo cubes, kept as rings of planes
  along block columns) on odd, even, ragged, walled and periodic lattices, with the
  halo-9 and halo-12 cubes: A_h against the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2005_12764_gb300 import inputs, serving

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


def test_chain_mode_walls_ragged_near_contact_matches_oracle(lbm):
    # 150 x 60 x 64: 5 x 8 tiles (ragged in x and y). The step kernel runs in chain
    # mode: 7 bands of 9 planes (one CTA per band and tile) and the top plane shared
    # by the 24 remaining CTAs, whose runs cross from one tile to the next.
    shape = (64, 60, 150)
    drops = [(20.0, 12.0, 30.0, 6.0), (33.5, 24.0, 31.0, 6.5), (50.0, 30.0, 50.0, 7.0),
             (110.0, 40.0, 20.0, 8.0), (130.0, 20.0, 55.0, 6.0)]
    rr, rb = inputs.paint_droplets(shape, drops, periodic=(True, False, False))
    kw = dict(wall_y=1, wall_z=1, sigma=0.02, beta=0.7, A_nc=0.02, h_min=3.0, g=(1e-5, 0, 0))
    nz, ny, nx = shape
    o = oracle.Lattice(oracle.make_params(nx, ny, nz, **kw))
    o.set_fields(rr, rb)
    o.step(30)
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, **kw))
    g.set_fields(rr, rb)
    g.step(30)
    fo, fg = o.get_fields(), g.get_fields()
    e = {k: float(np.abs(fo[k] - fg[k]).max()) for k in ("rho_r", "rho_b", "u")}
    assert e["rho_r"] <= RHO_TOL and e["rho_b"] <= RHO_TOL and e["u"] <= U_TOL, e
    g.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16", "fp32_q5", "fp16_q5"])
def test_chain_mode_is_bitwise_part_mode(lbm, storage):
    # A sheared 128^3 droplet: lbm_step runs chain mode (64 tiles: 4 bands of 28
    # planes and 16 planes shared by 48 CTAs), the serving engine part mode; every
    # node's update is computed the same way in both.
    req = dict(id=0, L=128, R=32.0, sigma=0.02, steps=24, sheared=True)
    p, rr, rb = serving.request_lattice(req, storage)
    g = lbm.Lattice(p)
    g.set_fields(rr, rb)
    g.step(req["steps"])
    f = g.get_fields()
    g.close()
    e = lbm.Engine(budget_bytes=8 << 30, max_slots=4, chunk_steps=10, autotune=False)
    t = e.submit(p, rr, rb, req["steps"])
    for _ in range(100):
        if e.state(t) in ("finished", "failed"):
            break
        e.tick()
    assert e.state(t) == "finished"
    res = e.result(t)
    e.close()
    for k in ("rho_r", "rho_b", "u", "phi"):
        assert np.array_equal(res[k], f[k]), k


BOUND_CASES = {
    "odd_walls_ragged": dict(shape=(13, 29, 45), walls=True,
                             drops=[(12.0, 10.0, 6.0, 5.0), (24.5, 18.0, 6.5, 5.5),
                                    (38.0, 9.0, 6.0, 4.5)]),
    "odd_periodic": dict(shape=(19, 21, 37), walls=False,
                         drops=[(10.0, 10.0, 9.0, 6.0), (25.0, 11.0, 10.0, 6.5),
                                (36.0, 3.0, 1.0, 4.0)]),
    "even_periodic": dict(shape=(24, 32, 48), walls=False,
                          drops=[(10.0, 16.0, 12.0, 7.0), (26.0, 15.0, 11.0, 7.5),
                                 (47.0, 31.0, 23.0, 5.0)]),
}


@pytest.mark.parametrize("case", sorted(BOUND_CASES))
def test_near_contact_pass_on_odd_ragged_lattices(lbm, case):
    # The near-contact pass works in 16 x 8 x 8 blocks with halo cubes (wrapped at
    # periodic seams, clamped at walls): on odd, ragged, walled and periodic lattices
    # every node's A_h equals the oracle's full ray march, after several steps
    # (threshold branches proven).
    import branch_cases
    c = BOUND_CASES[case]
    shape = c["shape"]
    nz, ny, nx = shape
    per = (True, not c["walls"], not c["walls"])
    rr, rb = inputs.paint_droplets(shape, c["drops"], periodic=per)
    kw = dict(sigma=0.02, beta=0.7, A_nc=0.02, h_min=3.0)
    if c["walls"]:
        kw.update(wall_y=1, wall_z=1)
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, **kw))
    g.set_fields(rr, rb)
    op = oracle.make_params(nx, ny, nz, **kw)
    seen = 0
    for steps in (1, 3, 10):
        g.step(steps)
        _, _, lag = g.get_pops()
        got = g.get_nc_field()
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    want = oracle.nc_strength_node(op, lag, x, y, z)
                    tol = 1e-6 * kw["A_nc"] + 1e-3 * abs(want)
                    if abs(got[z, y, x] - want) > tol:
                        assert branch_cases.ah_explained(
                            op, lag, x, y, z, got[z, y, x],
                            1e-6 * kw["A_nc"] + 1e-3 * abs(got[z, y, x])), (steps, x, y, z)
                    seen += want > 0
    assert seen > 50
    g.close()


SEGMENT_CASES = [("periodic", dict(h_min=3.0)), ("periodic_halo12", dict(h_min=4.0, h_cut=8.0)),
                 ("walls_halo12", dict(h_min=3.0, h_cut=9.0, wall_y=1, wall_z=1))]


@pytest.mark.parametrize("case", range(len(SEGMENT_CASES)), ids=[c[0] for c in SEGMENT_CASES])
def test_near_contact_pass_column_segments(lbm, case):
    # A lattice with enough block columns that the pass walks segments of several
    # blocks along z (its halo cube a ring of planes, each later block copying only the
    # planes that enter its window), with the halo-9 and halo-12 cubes (h_cut <= 6,
    # h_cut up to 9), periodic and walled: A_h at 40,000 random nodes and at up to
    # 40,000 nodes where the GPU measured a film equals the oracle's ray march
    # (threshold branches and ray directions rounded in FP32 proven).
    import branch_cases
    import torch
    name, extra = SEGMENT_CASES[case]
    nz, ny, nx = 128, 128, 256
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cols, bzn = (nx // 16) * (ny // 8), nz // 8
    assert min(16, bzn, cols * bzn // (8 * sms)) > 1      # segments of more than one block
    rng = np.random.default_rng(40 + case)
    drops = [(float(rng.uniform(0, nx)), float(rng.uniform(0, ny)), float(rng.uniform(0, nz)),
              float(rng.uniform(5.0, 8.0))) for _ in range(420)]
    walls = bool(extra.get("wall_y"))
    rr, rb = inputs.paint_droplets((nz, ny, nx), drops, periodic=(True, not walls, not walls))
    kw = dict(sigma=0.02, beta=0.7, A_nc=0.02, **extra)
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, **kw))
    g.set_fields(rr, rb)
    g.step(3)
    _, _, lag = g.get_pops()
    got = g.get_nc_field()
    op = oracle.make_params(nx, ny, nz, **kw)
    films = np.argwhere(got > 0)
    assert len(films) > 1000
    pick = rng.choice(len(films), size=min(len(films), 40000), replace=False)
    nodes = [tuple(v) for v in films[pick]]
    nodes += [(int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx)))
              for _ in range(40000)]
    lag = np.ascontiguousarray(lag, dtype=np.float64)
    G = oracle.gradient(op, lag)
    turned = 0
    for (z, y, x) in nodes:
        want = oracle.nc_strength_node(op, lag, x, y, z)
        tol = 1e-6 * kw["A_nc"] + 1e-3 * abs(want)
        if abs(got[z, y, x] - want) > tol:
            tg = 1e-6 * kw["A_nc"] + 1e-3 * abs(got[z, y, x])
            if branch_cases.ah_explained(op, lag, x, y, z, got[z, y, x], tg):
                continue
            # (a ray direction rounded differently in FP32, at a small |G'|)
            assert branch_cases.ah_direction_explained(op, lag, x, y, z, got[z, y, x], tg,
                                                       G[:, z, y, x]), \
                (name, x, y, z, got[z, y, x], want)
            turned += 1
    assert turned <= 1e-3 * len(nodes), turned
    g.close()
