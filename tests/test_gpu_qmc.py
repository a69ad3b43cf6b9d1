"""Parity of the FP64-class CUDA Hirsch-Fye paths with the CPU oracle, through the C ABI.

precision 0 = FP64 sweeps (the FP64 solver), precision 2 = FP32-pair sweeps (a 48-bit
significand between FP64 refreshes; not FP64 arithmetic).  Bar: identical accept decisions under
the same Philox stream (fields compared after every sweep) and G within 1e-10 of the oracle
relative to max|G| for both; measurement bins within 1e-10 for the FP64 form.  The pair form's
bins average G over the sweeps between refreshes, where its 48-bit updates drift further from
FP64 than FP64 itself does; they are held to 5e-10, its own bar, which is not an FP64 claim.
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


def _ctx(hf, **over):
    cfg = dict(wl.CONFIGS["square6"])
    cfg.update(over)
    return hf.Context(hf.make_params(cfg)), cfg


class OracleChain:
    def __init__(self, seed, site, ch, L, lam, gup, gdn, refresh_every, stagger=0):
        self.g0u, self.g0d = o.build_g0(gup), o.build_g0(gdn)
        self.s = o.init_fields(seed, site, ch, L)
        self.Gu, _ = o.dyson(self.g0u, self.s, 1, lam)
        self.Gd, _ = o.dyson(self.g0d, self.s, -1, lam)
        self.seed, self.site, self.ch, self.lam, self.re = seed, site, ch, lam, refresh_every
        self.phase = (site + ch) % refresh_every if (stagger and refresh_every > 0) else 0
        self.nsw = 0
        self.acc = 0
        self.meas = []

    def sweep(self, measure):
        self.acc += o.sweep(self.lam, self.seed, self.site, self.ch, self.nsw, self.s, self.Gu,
                            self.Gd)
        self.nsw += 1
        if self.re > 0 and (self.nsw + self.phase) % self.re == 0:
            self.Gu, _ = o.dyson(self.g0u, self.s, 1, self.lam)
            self.Gd, _ = o.dyson(self.g0d, self.s, -1, self.lam)
        if measure:
            self.meas.append(o.measure(self.Gu, self.Gd))


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_initial_fields_bit_exact(hf):
    ctx, cfg = _ctx(hf, chains_per_site=3, beta=8.0, dtau=0.25)
    f, cnt = hf.hf_get_fields(ctx.handle, ctx.n_chains, ctx.L)
    assert np.all(cnt == 0)
    for c in range(ctx.n_chains):
        site, ch = divmod(c, 3)
        assert np.array_equal(f[c], o.init_fields(cfg["seed"], site, ch, ctx.L))


@pytest.mark.parametrize("stagger", [0, 1])
@pytest.mark.parametrize("team_warps", [0, 2, 4])
@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("L,beta", [(8, 2.0), (12, 3.0), (16, 4.0), (20, 5.0), (24, 6.0),
                                    (32, 8.0), (40, 10.0), (48, 12.0), (64, 16.0)])
def test_sweeps_identical_decisions(hf, L, beta, precision, team_warps, stagger):
    cps, re, nsweep, bs = 2, 7, 24, 4
    ctx, cfg = _ctx(hf, chains_per_site=cps, beta=beta, dtau=0.25, U=6.0, refresh_every=re,
                    bin_size=bs, max_bins=nsweep // bs, seed=1234 + L, precision=precision,
                    team_warps=team_warps, refresh_stagger=stagger)
    assert ctx.L == L
    baths = wl.random_baths(L, ctx.n_sites, beta, L)
    for i in range(ctx.n_sites):
        for sp in range(2):
            hf.hf_set_g0(ctx.handle, i, sp, baths[i, sp])
    _, lam = o.constants(beta, 6.0, L)
    ref = [OracleChain(cfg["seed"], c // cps, c % cps, L, lam, baths[c // cps, 0],
                       baths[c // cps, 1], re, stagger) for c in range(ctx.n_chains)]
    for k in range(nsweep):
        hf.hf_sweep(ctx.handle, 0, 1, 1 if k == 0 else 0)
        fields, cnt = hf.hf_get_fields(ctx.handle, ctx.n_chains, L)
        for c, r in enumerate(ref):
            r.sweep(True)
            assert np.array_equal(fields[c], r.s), "decision mismatch: sweep %d chain %d" % (k, c)
        assert np.all(cnt == k + 1)
    acc = hf.hf_get_accepts(ctx.handle, ctx.n_chains)
    worst = 0.0
    for c, r in enumerate(ref):
        assert acc[c] == r.acc
        G = hf.hf_get_green(ctx.handle, c, L)
        worst = max(worst, _rel(G[0], r.Gu), _rel(G[1], r.Gd))
    assert worst < 1e-10, worst
    assert sum(r.acc for r in ref) > 0
    # bins -> per-site means and errors, oracle reduction done here by numpy
    for i in range(ctx.n_sites):
        gtau, n, d, m, errs = hf.hf_measure(ctx.handle, i, L)
        x = []
        for ch in range(cps):
            meas = np.array(ref[i * cps + ch].meas)
            x.append(meas.reshape(-1, bs, 2 * L + 3).sum(axis=1) / bs)
        x = np.concatenate(x)
        mean = x.mean(axis=0)
        err = x.std(axis=0, ddof=1) / np.sqrt(x.shape[0])
        # FP64 form: the FP64 bar; the 48-bit pair form: its own, looser bar (module docstring)
        tol = 1e-10 if precision == 0 else 5e-10
        assert np.abs(gtau - mean[:2 * L]).max() < tol
        assert abs(n[0] - mean[2 * L]) < tol and abs(n[1] - mean[2 * L + 1]) < tol
        assert abs(d - mean[2 * L + 2]) < tol
        assert abs(m - (mean[2 * L] - mean[2 * L + 1])) < tol
        assert np.abs(errs[:2 * L + 3] - err).max() < 10 * tol
    ctx.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_u0_is_bitwise_g0(hf, precision):
    # FP64 path: G = G0 bit for bit; FP32-pair path: G0 split into hi + lo (two 24-bit
    # truncations, relative error < 2^-46) and then left exactly unchanged by every (zero) update
    L, beta = 16, 4.0
    ctx, cfg = _ctx(hf, chains_per_site=2, U=0.0, beta=beta, dtau=0.25, refresh_every=3,
                    bin_size=5, max_bins=2, precision=precision)
    baths = wl.random_baths(99, ctx.n_sites, beta, L)
    for i in range(ctx.n_sites):
        for sp in range(2):
            hf.hf_set_g0(ctx.handle, i, sp, baths[i, sp])
    hf.hf_sweep(ctx.handle, 3, 7, 1)
    acc = hf.hf_get_accepts(ctx.handle, ctx.n_chains)
    assert np.all(acc == 10 * L)
    for c in range(ctx.n_chains):
        G = hf.hf_get_green(ctx.handle, c, L)
        site = c // 2
        for sp in range(2):
            g0 = o.build_g0(baths[site, sp])
            if precision == 0:
                assert np.array_equal(G[sp], g0)
            else:
                assert np.all(np.abs(G[sp] - g0) <= 2.0 ** -45 * np.abs(g0))
    ctx.close()


@pytest.mark.parametrize("precision,team_warps", [(0, 0), (2, 0), (2, 2), (2, 4)])
def test_full_size_batch_sampled_chains(hf, precision, team_warps):
    """The bench's workload shape (20x20 trap: 55 sites x 32 chains, L = 32) in the bench's
    launch configurations; a sample of chains is replayed by the oracle."""
    cfg = dict(wl.CONFIGS["square20"], n_warmup=6, n_measure=20, bin_size=10, max_bins=2,
               precision=precision, team_warps=team_warps)
    ctx = hf.Context(hf.make_params(cfg))
    L = ctx.L
    assert (ctx.n_sites, ctx.n_chains, L) == (55, 1760, 32)
    baths = wl.random_baths(2024, ctx.n_sites, cfg["beta"], L)
    for i in range(ctx.n_sites):
        for sp in range(2):
            hf.hf_set_g0(ctx.handle, i, sp, baths[i, sp])
    hf.hf_sweep(ctx.handle, 6, 20, 1)
    fields, cnt = hf.hf_get_fields(ctx.handle, ctx.n_chains, L)
    acc = hf.hf_get_accepts(ctx.handle, ctx.n_chains)
    assert np.all(cnt == 26)
    _, lam = o.constants(cfg["beta"], cfg["U"], L)
    for c in (0, 1, 31, 32, 777, 1000, 1728, 1759):
        site, ch = divmod(c, 32)
        r = OracleChain(cfg["seed"], site, ch, L, lam, baths[site, 0], baths[site, 1],
                        cfg["refresh_every"], cfg.get("refresh_stagger", 0))
        for k in range(26):
            r.sweep(k >= 6)
        assert np.array_equal(fields[c], r.s)
        assert acc[c] == r.acc
        G = hf.hf_get_green(ctx.handle, c, L)
        assert max(_rel(G[0], r.Gu), _rel(G[1], r.Gd)) < 1e-10
    ctx.close()


@pytest.mark.parametrize("L,beta,team_warps", [(8, 2.0, 1), (16, 4.0, 1), (20, 5.0, 1),
                                               (32, 8.0, 1)])
def test_delayed_updates_bitwise_equal_rank1(hf, L, beta, team_warps):
    """Rank-k delayed updates apply the same pair multiply-adds in the same order as rank-1
    updates, so every delay depth gives bit-for-bit the rank-1 result."""
    ref = None
    for k in (1, 4, 8, 16, 32):
        ctx, cfg = _ctx(hf, chains_per_site=2, beta=beta, dtau=0.25, U=7.0, refresh_every=5,
                        bin_size=4, max_bins=3, seed=77, precision=2, delay_k=k,
                        team_warps=team_warps)
        baths = wl.random_baths(3 * L, ctx.n_sites, beta, L)
        for i in range(ctx.n_sites):
            for sp in range(2):
                hf.hf_set_g0(ctx.handle, i, sp, baths[i, sp])
        hf.hf_sweep(ctx.handle, 3, 12, 1)
        out = (hf.hf_get_fields(ctx.handle, ctx.n_chains, L)[0],
               hf.hf_get_accepts(ctx.handle, ctx.n_chains),
               [hf.hf_get_green(ctx.handle, c, L) for c in (0, ctx.n_chains - 1)],
               [hf.hf_measure(ctx.handle, i, L)[0] for i in range(ctx.n_sites)])
        ctx.close()
        if ref is None:
            ref = out
            continue
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]), k
        for a, b in zip(out[2], ref[2]):
            assert np.array_equal(a, b), k
        for a, b in zip(out[3], ref[3]):
            assert np.array_equal(a, b), k


def test_resume_from_checkpoint_is_bitwise(hf):
    """Fields + sweep counters saved at a refresh boundary reproduce the uninterrupted run."""
    L, beta = 16, 4.0
    over = dict(chains_per_site=2, beta=beta, dtau=0.25, refresh_every=5, bin_size=5, max_bins=4)
    a, cfg = _ctx(hf, **over)
    b, _ = _ctx(hf, **over)
    baths = wl.random_baths(5, a.n_sites, beta, L)
    for ctx in (a, b):
        for i in range(ctx.n_sites):
            for sp in range(2):
                hf.hf_set_g0(ctx.handle, i, sp, baths[i, sp])
    hf.hf_sweep(a.handle, 20, 0, 1)
    hf.hf_sweep(b.handle, 10, 0, 1)
    f, cnt = hf.hf_get_fields(b.handle, b.n_chains, L)
    # a fresh context resumes from the checkpoint (counter 10 is a refresh boundary)
    c2, _ = _ctx(hf, **over)
    for i in range(c2.n_sites):
        for sp in range(2):
            hf.hf_set_g0(c2.handle, i, sp, baths[i, sp])
    hf.hf_set_fields(c2.handle, f, cnt)
    hf.hf_sweep(c2.handle, 10, 0, 1)
    fa, ca = hf.hf_get_fields(a.handle, a.n_chains, L)
    fc, cc = hf.hf_get_fields(c2.handle, c2.n_chains, L)
    assert np.array_equal(fa, fc) and np.array_equal(ca, cc)
    for c in range(a.n_chains):
        assert np.array_equal(hf.hf_get_green(a.handle, c, L), hf.hf_get_green(c2.handle, c, L))
    for ctx in (a, b, c2):
        ctx.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_zero_sweeps_is_a_pure_refresh(hf, precision):
    """hf_sweep with no sweeps and refresh_first = 1 leaves fields and counters alone and makes
    G the Dyson solution of the current fields (the empty launch)."""
    L, beta = 24, 6.0
    ctx, cfg = _ctx(hf, chains_per_site=2, beta=beta, dtau=0.25, U=5.0, precision=precision,
                    seed=99)
    baths = wl.random_baths(17, ctx.n_sites, beta, L)
    for i in range(ctx.n_sites):
        for sp in range(2):
            hf.hf_set_g0(ctx.handle, i, sp, baths[i, sp])
    f0, c0 = hf.hf_get_fields(ctx.handle, ctx.n_chains, L)
    hf.hf_sweep(ctx.handle, 0, 0, 1)
    f1, c1 = hf.hf_get_fields(ctx.handle, ctx.n_chains, L)
    assert np.array_equal(f0, f1) and np.array_equal(c0, c1) and np.all(c1 == 0)
    assert np.all(hf.hf_get_accepts(ctx.handle, ctx.n_chains) == 0)
    _, lam = o.constants(beta, 5.0, L)
    for c in range(ctx.n_chains):
        site = c // 2
        G = hf.hf_get_green(ctx.handle, c, L)
        for sp, sg in ((0, 1), (1, -1)):
            want, _ = o.dyson(o.build_g0(baths[site, sp]), f1[c], sg, lam)
            assert _rel(G[sp], want) < 1e-12
    ctx.close()
