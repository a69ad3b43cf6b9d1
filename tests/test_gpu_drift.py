"""The numerical-drift monitor (hf_params.check_drift): at every refresh inside a sweep launch the
kernels compare the state the Sherman-Morrison updates reached with the FP64 Dyson solution that
replaces it, and hf_get_drift reports the largest difference and the number of chain refreshes
checked.

Checked here, through the C ABI: the monitor changes nothing (fields, counters, G and bins are
bitwise those of a run without it); it counts exactly the in-launch refreshes (the refresh at a
launch's start is not checked); the drift it reports sits where each form's arithmetic puts it
(FP64 and FP32 pairs near rounding, FP32 several orders above); hf_clear_measurements resets it;
and with the monitor off it reads zero.
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


def _baths(ctx, hf, beta, L):
    b = wl.random_baths(11, ctx.n_sites, beta, L)
    for i in range(ctx.n_sites):
        for sp in range(2):
            hf.hf_set_g0(ctx.handle, i, sp, b[i, sp])


def _state(hf, ctx):
    f, cnt = hf.hf_get_fields(ctx.handle, ctx.n_chains, ctx.L)
    G = np.concatenate([hf.hf_get_green(ctx.handle, c, ctx.L).ravel() for c in range(ctx.n_chains)])
    return f, cnt, G


@pytest.mark.parametrize("precision,L,bound", [(0, 16, 1e-10), (2, 16, 1e-9), (2, 32, 1e-9),
                                               (0, 40, 1e-10)])
def test_drift_monitor_fused_forms(hf, precision, L, bound):
    cfg = dict(wl.CONFIGS["square6"], precision=precision, beta=L * 0.25, dtau=0.25,
               chains_per_site=3, n_warmup=10, n_measure=40, bin_size=10)
    out = {}
    for check in (0, 1):
        ctx = hf.Context(hf.make_params(dict(cfg, check_drift=check)))
        _baths(ctx, hf, cfg["beta"], ctx.L)
        hf.hf_sweep(ctx.handle, 10, 40, 1)      # refreshes after sweeps 10, 20, ..., 50
        hf.hf_sync(ctx.handle)
        out[check] = (_state(hf, ctx), hf.hf_get_drift(ctx.handle), ctx.n_chains)
        if check:
            hf.hf_clear_measurements(ctx.handle)
            assert hf.hf_get_drift(ctx.handle) == (0.0, 0)
        ctx.close()
    (f0, c0, G0), (d_off, n_off), nc = out[0]
    (f1, c1, G1), (d_on, n_on), _ = out[1]
    assert np.array_equal(f0, f1) and np.array_equal(c0, c1) and np.array_equal(G0, G1)
    assert (d_off, n_off) == (0.0, 0)
    assert n_on == 5 * nc
    assert 0.0 < d_on < bound


def test_drift_monitor_fp32_form(hf):
    cfg = dict(wl.CONFIGS["square6"], precision=1, beta=4.0, dtau=0.25, chains_per_site=2,
               n_warmup=5, n_measure=20, bin_size=5, refresh_every=1)
    ctx = hf.Context(hf.make_params(dict(cfg, check_drift=1)))
    _baths(ctx, hf, cfg["beta"], ctx.L)
    hf.hf_sweep(ctx.handle, 5, 20, 1)
    d, n = hf.hf_get_drift(ctx.handle)
    assert n == 25 * ctx.n_chains                  # every sweep ends with a checked refresh
    assert 1e-8 < d < 1e-2                         # single-precision updates drift visibly
    ctx.close()
