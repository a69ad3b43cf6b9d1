"""The numerical-drift monitor (hf_params.check_drift): at every refresh inside a sweep launch the
kernels compare the state the Sherman-Morrison updates reached with the FP64 Dyson solution that
replaces it, and hf_get_drift reports the largest difference and the number of chain refreshes
checked.

Checked here, through the C ABI:
- the monitor changes nothing: fields, counters and G are bitwise those of a run without it;
- it counts exactly the in-launch refreshes (the refresh at a launch's start is not checked);
- hf_clear_measurements resets it, and with the monitor off it reads zero;
- the drift it reports matches the oracle's. The oracle runs the same chains in FP64, with
  identical decisions, stops at each refresh point and compares with its own Dyson solve.
  - The FP64 form carries the same amplified rounding, in another order, so its value lies
    within a factor 10 of the oracle's.
  - A lazily normalised FP32 pair carries up to ~L 2^-48 relative error per update against
    FP64's 2^-53, a factor of at most 32 L. So the pair form lies between a tenth of the
    oracle's value and 10^4 times it.
"""
import numpy as np
import pytest

import oracle as o
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


BATH_SEED = 11


def _baths(ctx, hf, beta, L):
    b = wl.random_baths(BATH_SEED, ctx.n_sites, beta, L)
    for i in range(ctx.n_sites):
        for sp in range(2):
            hf.hf_set_g0(ctx.handle, i, sp, b[i, sp])


def _state(hf, ctx):
    f, cnt = hf.hf_get_fields(ctx.handle, ctx.n_chains, ctx.L)
    G = np.concatenate([hf.hf_get_green(ctx.handle, c, ctx.L).ravel() for c in range(ctx.n_chains)])
    return f, cnt, G


def _oracle_drift(L, beta, U, seed, cps, nsite, segments, per_segment):
    """Largest max |G_SM - G_Dyson| of the oracle's FP64 chains over the refreshes after each
    segment (the chains start from a Dyson solve, as a launch with refresh_first does)."""
    _, lam = o.constants(beta, U, L)
    baths = wl.random_baths(BATH_SEED, nsite, beta, L)
    worst = 0.0
    for site in range(nsite):
        g0u, g0d = o.build_g0(baths[site, 0]), o.build_g0(baths[site, 1])
        for ch in range(cps):
            s = o.init_fields(seed, site, ch, L)
            Gu, _ = o.dyson(g0u, s, 1, lam)
            Gd, _ = o.dyson(g0d, s, -1, lam)
            nsw = 0
            for _ in range(segments):
                bins = np.zeros((1, 2 * L + 3))
                _, nsw = o.run_chain(lam, g0u, g0d, seed, site, ch, nsw, per_segment, 0, 0, 1,
                                     s, Gu, Gd, bins)
                Du, _ = o.dyson(g0u, s, 1, lam)
                Dd, _ = o.dyson(g0d, s, -1, lam)
                worst = max(worst, np.abs(Gu - Du).max(), np.abs(Gd - Dd).max())
                Gu[:] = Du
                Gd[:] = Dd
    return worst


@pytest.mark.parametrize("precision,L", [(0, 16), (2, 16), (0, 32), (2, 32), (0, 40)])
def test_drift_monitor_fused_forms(hf, precision, L):
    beta = L * 0.25
    cfg = dict(wl.CONFIGS["square6"], precision=precision, beta=beta, dtau=0.25,
               chains_per_site=3, n_warmup=10, n_measure=40, bin_size=10)
    out = {}
    for check in (0, 1):
        ctx = hf.Context(hf.make_params(dict(cfg, check_drift=check)))
        _baths(ctx, hf, beta, ctx.L)
        hf.hf_sweep(ctx.handle, 10, 40, 1)      # refreshes after sweeps 10, 20, ..., 50
        hf.hf_sync(ctx.handle)
        out[check] = (_state(hf, ctx), hf.hf_get_drift(ctx.handle), ctx.n_chains, ctx.n_sites)
        if check:
            hf.hf_clear_measurements(ctx.handle)
            assert hf.hf_get_drift(ctx.handle) == (0.0, 0)
        ctx.close()
    (f0, c0, G0), (d_off, n_off), nc, ns = out[0]
    (f1, c1, G1), (d_on, n_on), _, _ = out[1]
    assert np.array_equal(f0, f1) and np.array_equal(c0, c1) and np.array_equal(G0, G1)
    assert (d_off, n_off) == (0.0, 0)
    assert n_on == 5 * nc
    d_or = _oracle_drift(L, beta, cfg["U"], cfg["seed"], 3, ns, 5, 10)
    assert d_or > 0.0
    if precision == 0:
        assert d_or / 10 < d_on < 10 * d_or, (d_on, d_or)
    else:
        assert d_or / 10 < d_on < 1e4 * d_or, (d_on, d_or)


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
