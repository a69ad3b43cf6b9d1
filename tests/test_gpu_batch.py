"""Batched (uneven-L, fused, graph-captured) execution must give bit-for-bit what each context
gives alone: the same kernel code runs each chain, only the launch grouping differs."""
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


BETAS = (5.0, 8.0, 10.0, 16.0)      # L = 20, 32, 40, 64 at dtau = 0.25


_STREAM = []


def _stream():
    import torch

    if not _STREAM:
        _STREAM.append(torch.cuda.Stream())
    return _STREAM[0]


def _ctxs(hf, precision, team_warps=0, **over):
    out = []
    for k, beta in enumerate(BETAS):
        cfg = dict(wl.CONFIGS["square6"], beta=beta, dtau=0.25, U=8.0, chains_per_site=3,
                   precision=precision, team_warps=(team_warps if beta * 4 <= 32 else 0),
                   seed=40 + k, n_warmup=4, n_measure=12, bin_size=4, max_bins=3)
        cfg.update(over)
        out.append((hf.Context(hf.make_params(cfg), stream=_stream()), cfg))
    return out


def _set_baths(hf, ctx, beta):
    L = ctx.L
    baths = wl.random_baths(int(beta * 10), ctx.n_sites, beta, L)
    for i in range(ctx.n_sites):
        for sp in range(2):
            hf.hf_set_g0(ctx.handle, i, sp, baths[i, sp])


@pytest.mark.parametrize("precision,team_warps", [(0, 0), (2, 0), (2, 2)])
def test_fused_uneven_L_sweeps_equal_separate(hf, precision, team_warps):
    alone = _ctxs(hf, precision, team_warps)
    fused = _ctxs(hf, precision, team_warps)
    for (a, cfg), (f, _) in zip(alone, fused):
        _set_baths(hf, a, cfg["beta"])
        _set_baths(hf, f, cfg["beta"])
    for a, _ in alone:
        hf.hf_sweep(a.handle, 5, 10, 1)
    b = hf.hf_batch_create([f.handle for f, _ in fused], 0)
    hf.hf_batch_sweep(b, 5, 10, 1)
    assert hf.hf_batch_elapsed(b) > 0
    for (a, _), (f, _) in zip(alone, fused):
        fa, ca = hf.hf_get_fields(a.handle, a.n_chains, a.L)
        ff, cf = hf.hf_get_fields(f.handle, f.n_chains, f.L)
        assert np.array_equal(fa, ff) and np.array_equal(ca, cf)
        assert np.array_equal(hf.hf_get_accepts(a.handle, a.n_chains),
                              hf.hf_get_accepts(f.handle, f.n_chains))
        for c in (0, a.n_chains - 1):
            assert np.array_equal(hf.hf_get_green(a.handle, c, a.L), hf.hf_get_green(f.handle, c, f.L))
        for i in range(a.n_sites):
            assert np.array_equal(hf.hf_measure(a.handle, i, a.L)[0], hf.hf_measure(f.handle, i, f.L)[0])
    hf.hf_batch_free(b)
    for c, _ in alone + fused:
        c.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_graph_captured_batched_iterations_equal_plain(hf, precision):
    over = dict(n_matsubara=64)
    alone = _ctxs(hf, precision, **over)
    fused = _ctxs(hf, precision, **over)
    b = hf.hf_batch_create([f.handle for f, _ in fused], 1)
    for it in range(3):          # plain first call, then capture + launch, then replay
        for a, _ in alone:
            hf.hf_rdmft_step(a.handle)
        ms = hf.hf_batch_rdmft_step(b)
        assert ms > 0
        for (a, _), (f, _) in zip(alone, fused):
            ns, nw, L = a.n_sites, a.nw, a.L
            assert np.array_equal(hf.hf_get_sigma(a.handle, ns, nw), hf.hf_get_sigma(f.handle, ns, nw))
            ma, ea = hf.hf_get_observables(a.handle, ns, L)
            mf, ef = hf.hf_get_observables(f.handle, ns, L)
            assert np.array_equal(ma, mf) and np.array_equal(ea, ef)
            assert np.array_equal(hf.hf_get_fields(a.handle, a.n_chains, L)[0],
                                  hf.hf_get_fields(f.handle, f.n_chains, L)[0])
    hf.hf_batch_free(b)
    for c, _ in alone + fused:
        c.close()


def test_batch_rejects_invalid_groups(hf):
    a = _ctxs(hf, 0)[0][0]
    c = _ctxs(hf, 2)[0][0]
    with pytest.raises(hf.HFError):
        hf.hf_batch_create([a.handle, c.handle], 0)      # mixed sweep forms
    with pytest.raises(hf.HFError):
        hf.hf_batch_create([a.handle, a.handle], 0)      # repeated context
    d = hf.Context(hf.make_params(dict(wl.CONFIGS["square6"], n_matsubara=8)))   # default stream
    with pytest.raises(hf.HFError) as e:
        hf.hf_batch_create([d.handle], 1)
    assert "non-default" in str(e.value)
    for x in (a, c, d):
        x.close()


def test_autotuner_picks_a_valid_configuration(hf):
    from paper_1006_2716_gb300 import autotune

    res = autotune.tune([20, 64], chains=64, sweeps=6, use_cache=False)
    for L, r in res.items():
        assert (r["precision"], r["team_warps"], r["delay_k"]) in autotune.candidates(L)
        assert r["ms_per_sweep"] == min(r["table"].values()) > 0
