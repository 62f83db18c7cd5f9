"""Deciding whether a GPU/oracle difference at a node is a threshold branch.

The reading of the near-contact force (Eq. 11) has two thresholds: a ray sample
carries a sign only if |phi| > 1e-5, and a node has a ray only if its lagged
colour gradient has |G'| >= 1e-3. The GPU evaluates the ray in FP32, the oracle in
FP64, on the same (FP32) lagged colour field. Where a sample or a gradient lies
within FP32 rounding of a threshold, the two may take different branches, and A_h
then differs by a finite amount. Such a node is not a parity failure; any other
difference is.

A difference is accepted only if the oracle, evaluated with a threshold moved by
its FP32 rounding bound, reproduces the GPU's A_h within the comparison's
tolerance (and, for a whole step, the oracle's step at that node with the GPU's
A_h reproduces the GPU's populations). The bounds:

- a ray sample: the trilinear interpolation of FP32 corners (7 lerps, each
  within 1.5 ulp of values |phi| <= 1) is within 7e-7 of its FP64 value; the
  sample position t n' (|t| <= 11) is within 2e-6 lattice units of the FP64 one,
  since n' comes from an FP32 gradient (relative error ~1e-7), and |grad phi| <=
  1 per lattice unit moves the value by at most as much. Bound: 3e-6.
- |G'|: 18 FP32 terms of magnitude <= 1/6, summed with FMAs, and a square root:
  within 5e-7. Bound: 1e-6.

The same rounding moves the ray: each component of G' (10 FMA terms) is within 1e-6
of its FP64 value, so where |G'| is small (it is >= 1e-3) the FP32 direction may
turn by up to about 1e-6/|G'|, the samples far along the ray move with it, and with
them the crossings and h. Such a difference is accepted only if the GPU's A_h lies
within the comparison's tolerance of the range of the oracle's A_h over the
gradients G' + (+-1e-6, +-1e-6, +-1e-6) (away from threshold branches A_h is
continuous in the direction, so every value between two of those is reached by a
gradient in that box).
"""
from __future__ import annotations

import numpy as np

import oracle

BAND, G_MIN = 1e-5, 1e-3
D_SAMPLE, D_GRAD = 3e-6, 1e-6


def ah_variants(P, lag, x, y, z, pin=None):
    """A_h of the reading at node (x, y, z) with each threshold at its value and
    moved down and up by its rounding bound (9 evaluations)."""
    return [oracle.nc_strength_node_thr(P, lag, x, y, z, band, g, pin)
            for band in (BAND - D_SAMPLE, BAND, BAND + D_SAMPLE)
            for g in (G_MIN - D_GRAD, G_MIN, G_MIN + D_GRAD)]


def ah_explained(P, lag, x, y, z, got, tol, pin=None) -> bool:
    """True if some threshold variant of the oracle's A_h is within tol of got."""
    return any(abs(v - got) <= tol for v in ah_variants(P, lag, x, y, z, pin))


def ah_direction_explained(P, lag, x, y, z, got, tol, G, pin=None) -> bool:
    """True if got lies within tol of the range of the oracle's A_h over the lagged
    gradients G + (+-D_GRAD, +-D_GRAD, +-D_GRAD) (G = the FP64 gradient at the node)."""
    vals = [oracle.nc_strength_node_g(P, lag, x, y, z,
                                      (G[0] + sx * D_GRAD, G[1] + sy * D_GRAD, G[2] + sz * D_GRAD),
                                      pin=pin)
            for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]
    return min(vals) - tol <= got <= max(vals) + tol


def step_explained(P, fr, fb, lag, node, got_r, got_b, ah_gpu, tol=1e-6, pin=None):
    """True if the GPU's A_h at flat node `node` is a threshold variant of the
    oracle's, and the oracle's step at that node with the GPU's A_h gives the GPU's
    populations (got_r, got_b: [19], oracle order) within tol."""
    nx, ny = P.nx, P.ny
    x, y, z = node % nx, (node // nx) % ny, node // (nx * ny)
    lag3 = np.asarray(lag).reshape(P.nz, P.ny, P.nx)
    if not ah_explained(P, lag3, x, y, z, ah_gpu, 1e-6 * P.A_nc + 1e-3 * abs(ah_gpu), pin):
        return False
    oa, ob, _ = oracle.step_nodes(P, fr, fb, lag, np.array([node]), pin=pin,
                                  ah=np.array([ah_gpu]))
    return bool(np.abs(oa[0] - got_r).max() <= tol and np.abs(ob[0] - got_b).max() <= tol)
