"""The allocation-free lattice step (for callers that cannot allocate device memory at call
time) must give what the workspace-backed lattice step of hf_rdmft_step gives, call after call.

Collected last on purpose: if it fails, a run that stops at the first failure has already run
every other test.  It passes alone in a fresh process and after the rest of the suite.
"""
import numpy as np
import pytest

from paper_1006_2716_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1006_2716_gb300 import build as B

    B.build()
    from paper_1006_2716_gb300 import hf as H

    return H


@pytest.mark.parametrize("form", [0, 1])
def test_noalloc_matches_workspace_lattice_step_twice(hf, form):
    import torch

    # the 20x20 trap: one band is 400 x 21 complex = 134 KB, so the 1000 (w_n, sigma) matrices
    # run in several chunks through the 16 MiB static array (form 1: blocked band form)
    cfg = dict(wl.CONFIGS["square20"], chains_per_site=1, n_warmup=2, n_measure=4, bin_size=2,
               max_bins=2, lattice_form=form)
    ctx = hf.Context(hf.make_params(cfg))
    ns, nw = ctx.n_sites, ctx.nw
    d_sigma = torch.empty((ns, 2, nw), dtype=torch.complex128, device="cuda")
    d_gloc = torch.empty((ns, 2, nw), dtype=torch.complex128, device="cuda")
    for call in range(2):
        # self-energy before this iteration; the iteration's own lattice phase uses it
        sigma = hf.hf_get_sigma(ctx.handle, ns, nw)
        hf.hf_rdmft_step(ctx.handle)
        want = hf.hf_get_gloc(ctx.handle, ns, nw)
        d_sigma.copy_(torch.from_numpy(sigma))
        d_gloc.fill_(float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        hf.hf_lattice_step_noalloc(ctx.handle, d_sigma.data_ptr(), d_gloc.data_ptr())
        free_after = torch.cuda.mem_get_info()[0]
        if call > 0:
            # the first call may load the module and look up the static array; from then on a
            # call must leave the device's free memory exactly as it found it (a cudaMalloc inside
            # the library would not show in torch's allocator statistics, but shows here)
            assert free_after == free_before, (free_before, free_after)
        got = d_gloc.cpu().numpy()
        assert np.all(np.isfinite(got)), "call %d left outputs unwritten" % call
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), "call %d" % call
    ctx.close()


def test_noalloc_rejects_oversized_band(hf):
    # disc of radius 60: 11 305 sites, band half-width 121 -> 22 MB per band > 16 MiB
    cfg = dict(wl.CONFIGS["square6"], Lx=60, geometry=1, n_matsubara=2, chains_per_site=1,
               n_warmup=1, n_measure=1, bin_size=1, max_bins=1)
    ctx = hf.Context(hf.make_params(cfg))
    import torch

    buf = torch.zeros((ctx.n_sites, 2, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(hf.HFError) as e:
        hf.hf_lattice_step_noalloc(ctx.handle, buf.data_ptr(), buf.data_ptr())
    assert e.value.status == hf.HF_EINVAL and "16777216" in str(e.value)
    ctx.close()
