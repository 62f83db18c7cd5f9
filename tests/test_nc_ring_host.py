"""The near-contact pass's ring of cube planes on the host: a block column walked in a
segment of blocks (NB_Z = 8 planes each) keeps the SZ planes of the current block's
window (halo H above and below) in a ring of SZ slots; the first block copies its whole
window, every later one only the NB_Z planes that enter it, into the slots of the NB_Z
that left. Restated here with plane numbers in place of colour values: after every
fill, window plane k of every block sits in slot (zbase + k) mod SZ, as the pass reads
it, for the halo-9 and halo-12 cubes and segments of any length."""
import pytest

NB_Z = 8


@pytest.mark.parametrize("H", [9, 12])
@pytest.mark.parametrize("seg", [1, 2, 3, 7, 16])
def test_ring_holds_every_window(H, seg):
    SZ = NB_Z + 2 * H
    ring = [None] * SZ
    zbase = 0
    z_first = 40
    for b in range(seg):
        z0 = z_first + b * NB_Z
        k0 = 0 if b == 0 else SZ - NB_Z
        for k in range(k0, SZ):                     # the fill: window plane k of this block
            ring[(zbase + k) % SZ] = z0 - H + k
        for k in range(SZ):                         # what the block reads
            assert ring[(zbase + k) % SZ] == z0 - H + k, (b, k)
        zbase = (zbase + NB_Z) % SZ                 # the next block's window starts NB_Z up
    # the incremental fills copy SZ + (seg - 1) NB_Z planes instead of seg SZ
    assert SZ + (seg - 1) * NB_Z <= seg * SZ
