"""The step kernel's work split (host logic; no device needed): every (tile, plane)
unit of a lattice is marched by exactly one CTA, in part mode and in chain mode, for
the documented splits of the benchmark and test lattices and for a spread of shapes
and GPU sizes. The assignment of units to CTAs is restated here from the rules that
include/lbm.h states for lbm_work_split."""
import math

import numpy as np
import pytest

from paper_2005_12764_gb300 import build_lib, lbm

TX, TY = 32, 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    build_lib.build()
    lbm.load()


def coverage(nx, ny, nz, w):
    """count[tile, z]: how many CTAs march unit (tile, z); tiles row-major, x fastest."""
    tx_n, ty_n = math.ceil(nx / TX), math.ceil(ny / TY)
    T = tx_n * ty_n
    count = np.zeros((T, nz), dtype=np.int64)
    if w["chain"] > 0:
        k, h = w["band_k"], w["band_h"]
        assert w["grid"] == w["chain"] and 1 <= k and k * h <= nz
        nfull, zr = k * T, k * h
        nr = nz - zr
        R = w["grid"] - nfull
        assert nr == 0 or R > 0
        for c in range(w["grid"]):
            if c < nfull:
                band, tile = divmod(c, T)
                count[tile, band * h:(band + 1) * h] += 1
            else:
                U = T * nr
                for u in range(U * (c - nfull) // R, U * (c - nfull + 1) // R):
                    t, z = divmod(u, nr)               # column-major tile order
                    txi, tyi = divmod(t, ty_n)
                    count[tyi * tx_n + txi, zr + z] += 1
    else:
        zp = w["zparts"]
        assert w["grid"] == T * zp
        for c in range(w["grid"]):
            part, tile = divmod(c, T)
            count[tile, nz * part // zp:nz * (part + 1) // zp] += 1
    return count


def split(nx, ny, nz, sms, **kw):
    return lbm.work_split(lbm.make_params(nx, ny, nz, **kw), sms)


@pytest.mark.parametrize("shape,want", [
    ((256, 128, 64), dict(chain=304, band_k=2, band_h=28)),    # the channel: 8 planes left
    ((150, 60, 64), dict(chain=304, band_k=7, band_h=9)),      # 40 tiles: 1 plane left
    ((128, 128, 128), dict(chain=304, band_k=4, band_h=28)),   # 64 tiles: 16 planes left
])
def test_documented_chain_splits_on_152_sms(shape, want):
    w = split(*shape, 152)
    for k, v in want.items():
        assert w[k] == v, (shape, w)
    assert (coverage(*shape, w) == 1).all()


def test_large_lattice_uses_part_mode():
    w = split(512, 512, 512, 152)       # 1024 tiles: more tiles than CTA slots
    assert w["chain"] == 0 and w["grid"] == 1024 * w["zparts"]
    assert (coverage(512, 512, 512, w) == 1).all()


@pytest.mark.parametrize("sms", [1, 7, 132, 152])
def test_every_unit_exactly_once(sms):
    rng = np.random.default_rng(sms)
    shapes = [(1, 1, 1), (4, 1, 1), (5, 3, 1), (2, 2, 2), (33, 9, 17), (64, 64, 64),
              (100, 50, 300), (40, 200, 31)]
    shapes += [tuple(int(v) for v in rng.integers(1, 200, size=3)) for _ in range(12)]
    for shape in shapes:
        w = split(*shape, sms)
        assert w["grid"] >= 1
        c = coverage(*shape, w)
        assert (c == 1).all(), (shape, sms, w)


def test_invalid_arguments_are_refused():
    with pytest.raises(lbm.LbmError):
        split(16, 16, 16, 0)
    with pytest.raises(lbm.LbmError):
        split(16, 16, 16, 152, tau_r=0.5)


@pytest.mark.parametrize("bad", [
    dict(storage=7), dict(storage="fp32_q5", model="shan_chen", G_sc=1.2),
    dict(storage="fp16_q5", model="shan_chen", G_sc=1.2), dict(storage="fp16_q5", rho0=0.0),
    dict(model="shan_chen", A_nc=0.01), dict(wall_u=0.01), dict(wall_y=1, wall_u=0.5),
    dict(beta=1.5), dict(sigma=-1.0), dict(A_nc=0.01, h_min=0.0), dict(A_nc=0.01, h_cut=12.0),
    dict(storage="fp16", rho0=0.0),
    dict(inplace=1, storage="fp32_q5"), dict(inplace=1, storage="fp16_q5"),
    dict(inplace=1, model="shan_chen", G_sc=1.2), dict(inplace=1, wall_y=1, wall_u=0.01),
    dict(inplace=3),
])
def test_parameter_validation_without_a_device(bad):
    # the parameter checks of lbm_create run before any device call; lbm_work_split
    # applies the same checks, so they are testable on the host
    with pytest.raises(lbm.LbmError):
        split(16, 16, 16, 152, **bad)


def test_inplace_block_index_limit():
    # in-place steps index a padded population block in 31 bits: 1290 x 1280 x 1280
    # FP32 (2.11e9 nodes, 2.16e9 padded positions per block) is refused in place and
    # accepted with two copies; 640^3 is accepted in place
    with pytest.raises(lbm.LbmError):
        split(1290, 1280, 1280, 152, inplace=1)
    split(1290, 1280, 1280, 152)
    split(640, 640, 640, 152, inplace=1, storage="fp16")
