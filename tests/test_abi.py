"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/lbm.h declares (no GPU needed: nothing here launches a kernel)."""
import os
import re

import numpy as np

import oracle
from paper_2005_12764_gb300 import build_lib, lbm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "lbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_library_builds_and_exports_header_symbols():
    build_lib.build()
    lib = lbm.load()
    decl = declared_functions()
    assert sorted(lbm.SYMBOLS) == decl
    for name in decl:
        assert hasattr(lib, name), name


def test_velocity_set_is_the_same_set_as_the_oracle():
    build_lib.build()
    c = lbm.velocity_set()
    co = oracle.lattice()[0]
    assert {tuple(v) for v in c} == {tuple(v) for v in co}
    for i in range(19):                       # documented order properties
        assert (c[18 - i] == -c[i]).all()
    assert (c[9] == 0).all()
    assert list(c[:, 2]) == sorted(c[:, 2])


def test_footprint_is_reported_without_a_device():
    build_lib.build()
    p = lbm.make_params(256, 128, 64)
    N = 256 * 128 * 64
    assert lbm.footprint_bytes(p) >= 2 * 2 * 19 * N * 4
    p16 = lbm.make_params(256, 128, 64, storage="fp16")
    assert lbm.footprint_bytes(p16) < lbm.footprint_bytes(p)
    # the reduced FP32 form: Q + 5 blocks per copy instead of 2Q
    p5 = lbm.make_params(256, 128, 64, storage="fp32_q5")
    full, red = lbm.footprint_bytes(p), lbm.footprint_bytes(p5)
    assert 2 * 24 * N * 4 <= red < full
    assert (full - red) >= 2 * (2 * 19 - 24) * N * 4
    # in place: one copy of the populations instead of two
    pa = lbm.make_params(256, 128, 64, storage="fp16", inplace=1)
    two, one = lbm.footprint_bytes(p16), lbm.footprint_bytes(pa)
    assert two - one >= 2 * 19 * N * 2 and one >= 2 * 19 * N * 2
