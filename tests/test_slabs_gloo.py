"""Z-slab domain decomposition on CPU: two (and three) gloo ranks each step their slab
of a lattice with the FP64 oracle and exchange halo planes through the library's
exchange logic; the owned planes must equal the whole-lattice oracle run bitwise.
Checks the decomposition (plane ranges, halo depth, wrapped local planes) and the
point-to-point exchange; the GPU side (lbm_get_planes / lbm_set_planes) is checked
in tests/test_gpu_slabs.py."""
import os
import socket

import numpy as np
import pytest

from paper_2005_12764_gb300 import slabs

Q = 19


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    from paper_2005_12764_gb300 import inputs
    shape = (30, 14, 16)        # (nz, ny, nx); walls along y, z periodic
    drops = [(5.0, 6.0, 7.0, 4.5), (11.0, 7.0, 13.0, 4.0), (7.5, 7.5, 24.0, 4.0),
             (12.0, 5.0, 1.5, 3.5)]
    rr, rb = inputs.paint_droplets(shape, drops, periodic=(True, False, True))
    kw = dict(wall_y=1, sigma=0.02, beta=0.7, A_nc=0.02, h_min=2.0, h_cut=4.0,
              kolmogorov_amp=1e-3, tau_r=0.9, tau_b=1.1)
    return shape, rr, rb, kw


def _oracle_slab_run(rank, world, dist, steps):
    """This rank's owned planes after `steps` steps of its slab (oracle stepping,
    library exchange)."""
    import torch
    import oracle
    shape, rr, rb, kw = _case()
    nz, ny, nx = shape
    H = slabs.halo_depth(kw["h_cut"])
    slabs.check(nz, world, H, False)
    z0, z1 = slabs.plane_ranges(nz, world)[rank]
    own = z1 - z0
    planes = slabs.local_planes(nz, world, rank, H)
    lat = oracle.Lattice(oracle.make_params(nx, ny, own + 2 * H, **kw))
    lat.set_fields(rr[planes], rb[planes])
    plane = nx * ny

    def pack(fr, fb, lag, a, b):   # planes a .. b-1 of (fr, fb, lag) as one vector
        return torch.from_numpy(np.concatenate([fr[:, a:b].ravel(), fb[:, a:b].ravel(),
                                                lag[a:b].ravel()]))

    for _ in range(steps):
        lat.step(1)
        fr, fb = lat.get_pops()
        lag = lat.get_phi_lag()
        b_own, t_own = pack(fr, fb, lag, H, 2 * H), pack(fr, fb, lag, own, own + H)
        b_halo, t_halo = torch.empty_like(b_own), torch.empty_like(t_own)
        slabs.exchange(b_own, t_own, b_halo, t_halo, rank, world, dist)
        n = Q * H * plane
        for buf, a in ((b_halo, 0), (t_halo, own + H)):
            v = buf.numpy()
            fr[:, a:a + H] = v[:n].reshape(Q, H, ny, nx)
            fb[:, a:a + H] = v[n:2 * n].reshape(Q, H, ny, nx)
            lag[a:a + H] = v[2 * n:].reshape(H, ny, nx)
        lat.set_pops(fr, fb, lag)
    fr, fb = lat.get_pops()
    return fr[:, H:H + own], fb[:, H:H + own]


def _worker(rank, world, port, steps, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, _oracle_slab_run(rank, world, dist, steps)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_equal_the_whole_lattice_bitwise(world):
    import torch.multiprocessing as mp
    import oracle
    steps = 6
    shape, rr, rb, kw = _case()
    nz, ny, nx = shape
    whole = oracle.Lattice(oracle.make_params(nx, ny, nz, **kw))
    whole.set_fields(rr, rb)
    whole.step(steps)
    wr, wb = whole.get_pops()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (z0, z1) in enumerate(slabs.plane_ranges(nz, world)):
        fr, fb = got[r]
        assert np.array_equal(fr, wr[:, z0:z1]) and np.array_equal(fb, wb[:, z0:z1]), r
    # the near-contact force acted (films between the droplets, A_h > 0 somewhere)
    lag = whole.get_phi_lag()
    P = oracle.make_params(nx, ny, nz, **kw)
    assert any(oracle.nc_strength_node(P, lag, x, y, z) > 0
               for z in range(nz) for y in range(ny) for x in range(nx))


def test_one_rank_is_its_own_neighbour():
    # world 1: the exchange wraps the slab onto itself (a periodic lattice with halos)
    import oracle
    shape, rr, rb, kw = _case()
    nz, ny, nx = shape
    whole = oracle.Lattice(oracle.make_params(nx, ny, nz, **kw))
    whole.set_fields(rr, rb)
    whole.step(4)
    wr, wb = whole.get_pops()
    fr, fb = _oracle_slab_run(0, 1, None, 4)
    assert np.array_equal(fr, wr) and np.array_equal(fb, wb)


def test_decomposition_host_logic():
    assert slabs.halo_depth(6.0) == 9 and slabs.halo_depth(0.5) == 3 and slabs.halo_depth(9.0) == 12
    r = slabs.plane_ranges(10, 3)
    assert r == [(0, 3), (3, 6), (6, 10)]
    assert slabs.local_planes(10, 3, 0, 2) == [8, 9, 0, 1, 2, 3, 4]
    assert slabs.local_planes(10, 3, 2, 2) == [4, 5, 6, 7, 8, 9, 0, 1]
    with pytest.raises(ValueError):
        slabs.check(10, 3, 4, False)        # 3 planes per rank < 4 halo planes
    with pytest.raises(ValueError):
        slabs.check(40, 2, 4, True)         # walls at the z extremes
