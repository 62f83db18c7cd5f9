"""Diagnostics of the paper's workloads, as plain definitions (test infrastructure).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the GPU library computes the
same quantities in its own kernels; these are the references they are checked
against.

- Droplet census (the dense-emulsion workload reports the number of droplets and
  their size distribution): the connected components of the set {phi > 0} under
  26-connectivity (nodes sharing a face, an edge or a corner), wrapping around
  periodic axes and not across walls. Component sizes are node counts. The
  definition is evaluated with a library primitive: the connected components of the
  graph whose edges join neighbouring positive nodes (scipy.sparse.csgraph).
- Structure factor (the gel workload reports the peak of S(k, t)): the radially
  averaged power spectrum of the colour-field fluctuation,
      S(k_b) = sum over modes m in shell b of |phi_hat(m)|^2 / (N * modes in shell b),
      phi_hat(m) = sum_x (phi(x) - mean phi) exp(-i k(m).x),
  k(m) = 2 pi (m_x/n_x, m_y/n_y, m_z/n_z) with m the signed mode indices, shell
  b = round(|k(m)| / dk), dk = 2 pi / max(n_x, n_y, n_z). The FFT is numpy's.
"""
from __future__ import annotations

import numpy as np


def droplets(phi, periodic=(True, True, True)):
    """(number of components, sizes sorted in descending order) of {phi > 0};
    phi is [z, y, x]; periodic = (x, y, z) axes that wrap."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    pos = np.asarray(phi) > 0.0
    nz, ny, nx = pos.shape
    idx = np.arange(pos.size).reshape(pos.shape)
    rows, cols = [], []
    # 13 of the 26 neighbour offsets (one of each opposite pair)
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if (dz, dy, dx) > (0, 0, 0)]
    z, y, x = np.nonzero(pos)
    for dx, dy, dz in offs:
        xs, ys, zs = x + dx, y + dy, z + dz
        ok = np.ones(x.shape, dtype=bool)
        for a, n, per in ((xs, nx, periodic[0]), (ys, ny, periodic[1]), (zs, nz, periodic[2])):
            if per:
                a %= n
            else:
                ok &= (a >= 0) & (a < n)
        xs, ys, zs = xs[ok], ys[ok], zs[ok]
        src = idx[z[ok], y[ok], x[ok]]
        nb = pos[zs, ys, xs]
        rows.append(src[nb])
        cols.append(idx[zs, ys, xs][nb])
    r = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    g = coo_matrix((np.ones(r.size), (r, c)), shape=(pos.size, pos.size)).tocsr()
    _, lab = connected_components(g, directed=False)
    lab = lab[pos.ravel()]
    if lab.size == 0:
        return 0, np.zeros(0, dtype=np.int64)
    sizes = np.bincount(lab)
    sizes = np.sort(sizes[sizes > 0])[::-1]
    return int(sizes.size), sizes.astype(np.int64)


def structure_factor(phi, nbins):
    """(k_b [nbins], S [nbins], modes [nbins]) of the definition above; phi is
    [z, y, x]. Shells with no modes have S = 0."""
    phi = np.asarray(phi, dtype=np.float64)
    nz, ny, nx = phi.shape
    N = phi.size
    F = np.fft.fftn(phi - phi.mean())
    P = (F * np.conj(F)).real
    def modes(n):
        m = np.arange(n, dtype=np.float64)
        m[m >= (n + 1) // 2] -= n           # signed mode indices, FFT order
        return m
    mz = modes(nz)[:, None, None]
    my = modes(ny)[None, :, None]
    mx = modes(nx)[None, None, :]
    k = 2 * np.pi * np.sqrt((mx / nx) ** 2 + (my / ny) ** 2 + (mz / nz) ** 2)
    dk = 2 * np.pi / max(nx, ny, nz)
    b = np.rint(k / dk).astype(np.int64)
    keep = b < nbins
    S = np.bincount(b[keep], weights=P[keep], minlength=nbins)
    cnt = np.bincount(b[keep], minlength=nbins)
    with np.errstate(invalid="ignore", divide="ignore"):
        S = np.where(cnt > 0, S / (N * np.maximum(cnt, 1)), 0.0)
    return dk * np.arange(nbins), S, cnt
