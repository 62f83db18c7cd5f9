"""Z-slab domain decomposition of one lattice over several ranks, one GPU each.

The paper runs its lattice codes with MPI domain decomposition of the fluid (Sec.
"High-performance LB code for bijel materials"): every process owns a part of the
lattice and exchanges first-neighbour data with the others each step. Here the
lattice is cut along z, which must be periodic (walls at the z extremes would belong
to the end ranks only). Rank r owns planes [z0_r, z1_r) and holds a local lattice of
those planes plus H halo planes on each side, periodic in z as a lattice of its own.

One step changes a node from data at most R planes away: the pull reads the
neighbouring planes, the colour gradient the colour field of the neighbouring planes
(hence their pulls, two planes), and the near-contact film measurement reads the
lagged colour field up to floor(h_cut) + 3 planes away (the farthest trilinear
corner of a ray sample at t <= h_cut + 2). With H = max(2, floor(h_cut) + 3) every
owned node of a local step is computed from correct data, exactly as in the whole
lattice, provided the halo planes hold the neighbours' state before the step. So
after each step the H owned planes at each end of a slab are sent to the neighbour,
which stores them as its halo: one exchange of 2H planes of stored state per rank
and step, bitwise in every storage format (lbm_get_planes / lbm_set_planes). The
halo planes are stepped too (redundant work, 2H planes per rank), which removes
any exchange inside the step. The collectives carry lattice state between point-
to-point neighbours only.
"""
from __future__ import annotations

import math


def halo_depth(h_cut: float) -> int:
    """Halo planes per side: the reach of one step (near-contact rays, gradient)."""
    return max(2, int(math.floor(h_cut)) + 3)


def plane_ranges(nz: int, world: int):
    """[(z0, z1)] owned by each rank: contiguous, sizes differing by one at most."""
    return [(nz * r // world, nz * (r + 1) // world) for r in range(world)]


def local_planes(nz: int, world: int, rank: int, H: int):
    """Global plane of each local plane of rank `rank` (halo below, owned, halo above),
    wrapped around the periodic z axis."""
    z0, z1 = plane_ranges(nz, world)[rank]
    return [(z % nz) for z in range(z0 - H, z1 + H)]


def check(nz: int, world: int, H: int, wall_z: bool):
    if wall_z:
        raise ValueError("slab decomposition needs a periodic z axis")
    own = min(z1 - z0 for z0, z1 in plane_ranges(nz, world))
    if own < H:
        raise ValueError(f"each rank needs at least {H} planes (halo depth); nz={nz}, "
                         f"ranks={world}")


def exchange(bottom_own, top_own, bottom_halo, top_halo, rank, world, dist=None):
    """Sends this rank's lowest owned planes (bottom_own) to the rank below and its
    highest (top_own) to the rank above, and receives the halos: bottom_halo from the
    rank below (its top_own), top_halo from the rank above (its bottom_own). Tensors
    of equal size on every rank (torch; CUDA with NCCL, CPU with gloo). With one rank
    the slab is its own neighbour on both sides."""
    if world == 1 or dist is None:
        bottom_halo.copy_(top_own)
        top_halo.copy_(bottom_own)
        return
    below, above = (rank - 1) % world, (rank + 1) % world
    # two rounds, so that messages between the same pair of ranks (both neighbours
    # are one rank when world == 2) cannot be matched out of order: upward (top_own
    # to the rank above, bottom_halo from the rank below), then downward
    for send, to, recv, frm in ((top_own, above, bottom_halo, below),
                                (bottom_own, below, top_halo, above)):
        ops = [dist.P2POp(dist.isend, send, to), dist.P2POp(dist.irecv, recv, frm)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class SlabLattice:
    """One rank's slab of a lattice on its GPU: a lbm.Lattice of the owned planes and
    the halos, stepped with a halo exchange after every step."""

    def __init__(self, lbm, nx, ny, nz, rank, world, dist=None, device="cuda", **params):
        import torch
        self.H = halo_depth(params.get("h_cut") or 2.0 * params.get("h_min", 3.0))
        check(nz, world, self.H, bool(params.get("wall_z", 0)))
        self.rank, self.world, self.dist = rank, world, dist
        self.z0, self.z1 = plane_ranges(nz, world)[rank]
        self.own = self.z1 - self.z0
        self.planes = local_planes(nz, world, rank, self.H)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.lat = lbm.Lattice(lbm.make_params(nx, ny, self.own + 2 * self.H, **params))
        nb = self.lat.planes_bytes(self.H)
        self.buf = [torch.empty(nb, dtype=torch.uint8, device=device) for _ in range(4)]

    def _local(self, a):
        """The local planes of a whole-lattice [.., nz, ny, nx] array."""
        return a[..., self.planes, :, :]

    def set_fields(self, rho_r, rho_b, u=None, pins=None):
        """Initial fields given for the whole lattice (host arrays)."""
        import numpy as np
        self.lat.set_fields(np.ascontiguousarray(self._local(rho_r)),
                            np.ascontiguousarray(self._local(rho_b)),
                            None if u is None else np.ascontiguousarray(self._local(u)))
        if pins is not None:
            self.lat.set_pin_mask(np.ascontiguousarray(self._local(pins)))

    def step_and_pack(self):
        """One local step, then the owned end planes into the send buffers."""
        H, own = self.H, self.own
        self.lat.step(1)
        self.lat.get_planes(H, H, self.buf[0])
        self.lat.get_planes(own, H, self.buf[1])
        self.lat.sync()

    def unpack(self):
        """The received halo planes into the local lattice."""
        self.lat.set_planes(0, self.H, self.buf[2])
        self.lat.set_planes(self.own + self.H, self.H, self.buf[3])

    def step(self, n=1):
        import torch
        b_own, t_own, b_halo, t_halo = self.buf
        for _ in range(n):
            self.step_and_pack()
            exchange(b_own, t_own, b_halo, t_halo, self.rank, self.world, self.dist)
            if b_halo.is_cuda:
                torch.cuda.synchronize(b_halo.device)   # received before the lattice reads it
            self.unpack()

    def get_fields(self):
        """Fields of the owned planes ([own, ny, nx] arrays)."""
        f = self.lat.get_fields()
        sl = slice(self.H, self.H + self.own)
        return {k: (v[:, sl] if k == "u" else v[sl]) for k, v in f.items()}

    def close(self):
        self.lat.close()


def step_slabs(slab_list, n=1):
    """Steps the slabs of one lattice held by one process (ranks 0 .. len - 1, e.g. on
    one GPU), exchanging their halos by device copies between the steps."""
    import torch
    w = len(slab_list)
    for _ in range(n):
        for sl in slab_list:
            sl.step_and_pack()
        for r, sl in enumerate(slab_list):
            sl.buf[2].copy_(slab_list[(r - 1) % w].buf[1])   # bottom halo <- below's top
            sl.buf[3].copy_(slab_list[(r + 1) % w].buf[0])   # top halo <- above's bottom
        torch.cuda.synchronize()
        for sl in slab_list:
            sl.unpack()
