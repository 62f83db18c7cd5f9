"""Z-slab decomposition on the GPU: the slabs of one lattice, each a context of its
owned planes plus halos, stepped on one GPU with their halos exchanged by device copies
between steps (lbm_get_planes / lbm_set_planes, the same state a multi-GPU run sends),
equal the whole lattice bitwise in every storage format. (The distributed exchange
itself is checked on CPU with gloo ranks in tests/test_slabs_gloo.py.)"""
import numpy as np
import pytest

from paper_2005_12764_gb300 import inputs, slabs

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


@pytest.mark.parametrize("storage,world", [("fp32", 2), ("fp32", 3), ("fp16", 2), ("fp32_q5", 2),
                                           ("fp16_q5", 2)])
def test_slabs_equal_the_whole_lattice_bitwise(lbm, storage, world):
    nz, ny, nx = 60, 40, 48
    w = inputs.dense_emulsion(L=48, volume_fraction=0.3, r_range=(4.0, 7.0), seed=21)
    drops = [d for d in w.droplets if d[1] < ny - 1]
    rr, rb = inputs.paint_droplets((nz, ny, nx), drops, periodic=(True, False, True))
    kw = dict(wall_y=1, sigma=0.01, beta=0.7, A_nc=0.01, h_min=3.0, kolmogorov_amp=1e-4,
              storage=storage)
    steps = 12
    whole = lbm.Lattice(lbm.make_params(nx, ny, nz, **kw))
    whole.set_fields(rr, rb)
    whole.step(steps)
    fw = whole.get_fields()
    whole.close()
    parts = [slabs.SlabLattice(lbm, nx, ny, nz, r, world, **kw) for r in range(world)]
    for sl in parts:
        sl.set_fields(rr, rb)
    slabs.step_slabs(parts, steps)
    for sl in parts:
        f = sl.get_fields()
        for k in ("rho_r", "rho_b", "phi"):
            assert np.array_equal(f[k], fw[k][sl.z0:sl.z1]), (k, sl.rank)
        assert np.array_equal(f["u"], fw["u"][:, sl.z0:sl.z1]), sl.rank
        sl.close()
