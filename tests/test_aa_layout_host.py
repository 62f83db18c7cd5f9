"""In-place (AA) storage on the host: the two alternating slot layouts and the read
and write rules of the in-place step, restated here, moving populations exactly as
two-copy pull streaming with halfway bounce-back does, over odd and even step counts,
with walls and periodic axes. The collision is replaced by a fixed random linear map
per node, so that every direction's slot matters. (The GPU kernels that follow these
rules are checked against the two-copy path and the oracle in tests/test_gpu_inplace.py.)
"""
import numpy as np
import pytest

import oracle

C = oracle.lattice()[0].astype(int)       # [19, 3] (c_x, c_y, c_z)
Q = len(C)
OPP = np.array([int(np.nonzero((C == -C[i]).all(1))[0][0]) for i in range(Q)])


def neighbour(x, y, z, c, shape, walls):
    """(x, y, z) + c wrapped on periodic axes, or None beyond a wall."""
    nz, ny, nx = shape
    xn, yn, zn = x + c[0], y + c[1], z + c[2]
    if (walls[0] and not 0 <= yn < ny) or (walls[1] and not 0 <= zn < nz):
        return None
    return xn % nx, yn % ny, zn % nz


def collide(f, M):
    return np.einsum("ij,jzyx->izyx", M, f)


def step_two_copy(f, M, shape, walls):
    nz, ny, nx = shape
    g = np.empty_like(f)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for i in range(Q):
                    s = neighbour(x, y, z, -C[i], shape, walls)
                    g[i, z, y, x] = f[i, s[2], s[1], s[0]] if s else f[OPP[i], z, y, x]
    return collide(g, M)


def slot(layout, i, x, y, z, shape, walls):
    """Where f*_i(x) sits: layout 0 (opp(i), x); layout 1 (i, x + c_i), or (opp(i), x)
    when x + c_i lies beyond a wall."""
    if layout == 1:
        n = neighbour(x, y, z, C[i], shape, walls)
        if n:
            return i, n
    return OPP[i], (x, y, z)


def step_in_place(A, layout, M, shape, walls):
    nz, ny, nx = shape
    f = np.empty_like(A)
    reads = set()
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for i in range(Q):
                    s = neighbour(x, y, z, -C[i], shape, walls)
                    if layout == 1:            # streamed already: the node's own slot
                        d, (xs, ys, zs) = i, (x, y, z)
                    elif s:                    # f*_i of x - c_i in its slot (opp(i), x - c_i)
                        d, (xs, ys, zs) = OPP[i], s
                    else:                      # from beyond a wall: f*_opp(i)(x) in (i, x)
                        d, (xs, ys, zs) = i, (x, y, z)
                    f[i, z, y, x] = A[d, zs, ys, xs]
                    reads.add((d, xs, ys, zs, x, y, z))
    g = collide(f, M)
    out = 1 - layout
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for i in range(Q):
                    d, (xs, ys, zs) = slot(out, i, x, y, z, shape, walls)
                    # every node writes only the slots it read (no two nodes race)
                    assert (d, xs, ys, zs, x, y, z) in reads
                    A[d, zs, ys, xs] = g[i, z, y, x]
    return out


def decode(A, layout, shape, walls):
    nz, ny, nx = shape
    f = np.empty_like(A)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                for i in range(Q):
                    d, (xs, ys, zs) = slot(layout, i, x, y, z, shape, walls)
                    f[i, z, y, x] = A[d, zs, ys, xs]
    return f


@pytest.mark.parametrize("shape,walls", [((3, 4, 5), (False, False)), ((4, 3, 5), (True, False)),
                                         ((4, 5, 3), (True, True)), ((1, 2, 3), (False, True))])
def test_in_place_layouts_move_populations_as_pull_streaming(shape, walls):
    rng = np.random.default_rng(sum(shape))
    M = np.eye(Q) + 0.1 * rng.standard_normal((Q, Q))
    f0 = rng.standard_normal((Q,) + shape)
    f = f0.copy()
    A = np.empty_like(f0)
    nz, ny, nx = shape
    for z in range(nz):                        # the initial state in layout 0
        for y in range(ny):
            for x in range(nx):
                for i in range(Q):
                    A[OPP[i], z, y, x] = f0[i, z, y, x]
    layout = 0
    for step in range(1, 6):
        f = step_two_copy(f, M, shape, walls)
        layout = step_in_place(A, layout, M, shape, walls)
        assert layout == step % 2
        assert np.allclose(decode(A, layout, shape, walls), f, rtol=0, atol=1e-12), step
