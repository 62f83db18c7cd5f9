"""The allocation-free totals entry point (lbm_totals_noalloc) against the
context-based reduction (lbm_observables), through the C-ABI.

Collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test. It must pass alone in a fresh process and after the
other tests (it keeps no state between calls that its result depends on).
"""
import numpy as np
import pytest

from paper_2005_12764_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_totals_without_allocation_match_observables_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12764_gb300 import build_lib, lbm
    build_lib.build()
    w = inputs.channel_droplets(nx=64, ny=40, nz=24, n_grid=(2, 2, 1), r_range=(4, 6), seed=5)
    nz, ny, nx = w.shape
    n = nx * ny * nz
    g = lbm.Lattice(lbm.make_params(nx, ny, nz, **w.params))
    g.set_fields(w.rho_r, w.rho_b)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                       # two calls in a row, different states
        g.step(7)
        fr, fb, _ = g.get_pops()
        # the library stores FP32, so these float64 values convert back exactly
        pops = torch.from_numpy(np.concatenate([fr.reshape(19, n), fb.reshape(19, n)])
                                .astype(np.float32)).cuda()
        out.fill_(-1.0)
        lbm.totals_noalloc(pops.data_ptr(), n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        got = out[:5].cpu().numpy()
        want = g.observables()[:5]
        mass = want[0] + want[1]
        # same FP32 values summed in FP64 in a different order
        assert np.allclose(got, want, rtol=1e-12, atol=1e-12 * mass), (call, got, want)
        assert (out[5:] == -1.0).all()          # nothing written past the 5 results


def test_totals_without_allocation_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12764_gb300 import build_lib, lbm
    build_lib.build()
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    pops = torch.zeros(38, dtype=torch.float32, device="cuda")
    for bad in (0, 512 ** 3 + 1):
        with pytest.raises(lbm.LbmError) as ei:
            lbm.totals_noalloc(pops.data_ptr(), bad, out.data_ptr())
        assert ei.value.status == -1


def test_totals_without_allocation_on_3m_nodes_with_a_ragged_last_block():
    # 3,000,017 nodes: 367 blocks of 8192 nodes, the last one holding 1695; random
    # FP32 populations summed by torch in FP64 per direction (a different order)
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_12764_gb300 import build_lib, lbm
    build_lib.build()
    c = torch.from_numpy(lbm.velocity_set().astype(np.float64)).cuda()     # [19, 3]
    gen = torch.Generator(device="cuda").manual_seed(2005)
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    for n in (3_000_017, 8192 * 5, 1):          # ragged, whole blocks only, one node
        pops = torch.rand(2 * 19, n, dtype=torch.float32, device="cuda", generator=gen) * 0.1
        out.fill_(-1.0)
        lbm.totals_noalloc(pops.data_ptr(), n, out.data_ptr())
        torch.cuda.synchronize()
        per_dir = pops.double().sum(dim=1)                               # [38]
        r, b = per_dir[:19], per_dir[19:]
        want = torch.cat([r.sum().view(1), b.sum().view(1), ((r + b)[:, None] * c).sum(0)])
        mass = float(want[0] + want[1])
        assert torch.allclose(out[:5], want, rtol=1e-12, atol=1e-12 * mass), (n, out[:5], want)
        assert (out[5:] == -1.0).all()
        del pops
