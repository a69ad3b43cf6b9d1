"""Parity of the FP64 sweep form at the benchmark's own scale and length, and the Lambda = 8
brute-force check of the 6x6 configuration through the CUDA path.

* The 20x20 trap (55 inequivalent sites x 32 chains, L = 32) runs one whole 2500-sweep launch
  (500 warm-up + 2000 measured, refresh every 10 sweeps: the QMC phase of one benchmark
  iteration) on the baths its own lattice step gives.  The same sweeps run again as 250 launches
  of 10 sweeps, whose fields are compared with the oracle's after every refresh on a sample of
  chains; the two device runs must end bit for bit in the same state, so the single launch took
  the oracle's decisions all along.  G and the bins of the sample are compared with the oracle at
  1e-10.  The oracle counts the near ties |u - R_up R_dn| < 1e-9 R_up R_dn it met: the proposals
  on which two correct FP64 implementations that round differently could decide differently.
* The 6x6 trap at dtau = 0.5 (L = 8): G(tau), densities and double occupancy of two impurities
  against the exact enumeration of all 2^8 Ising configurations.
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


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _state(hf, ctx):
    f, cnt = hf.hf_get_fields(ctx.handle, ctx.n_chains, ctx.L)
    return f, cnt, hf.hf_get_accepts(ctx.handle, ctx.n_chains)


def test_square20_whole_launch_identical_decisions(hf):
    cfg = dict(wl.CONFIGS["square20"], precision=0, team_warps=1)
    nwu, nme, re, bs = cfg["n_warmup"], cfg["n_measure"], cfg["refresh_every"], cfg["bin_size"]
    one = hf.Context(hf.make_params(cfg))
    L, ns, nc, cps = one.L, one.n_sites, one.n_chains, cfg["chains_per_site"]
    assert (ns, nc, L) == (55, 1760, 32)
    hf.hf_compute_baths(one.handle)
    g0 = hf.hf_get_g0(one.handle, ns, L)
    # (1) the benchmark's launch: every sweep of the iteration in one kernel launch
    hf.hf_sweep(one.handle, nwu, nme, 1)
    f1, c1, a1 = _state(hf, one)
    assert np.all(c1 == nwu + nme)
    # (2) the same sweeps as launches of one refresh interval each
    split = hf.Context(hf.make_params(cfg))
    for i in range(ns):
        for sp in range(2):
            hf.hf_set_g0(split.handle, i, sp, g0[i, sp])
    _, lam = o.constants(cfg["beta"], cfg["U"], L)
    sample = [0, 33, 64 + 5, 300, 577, 901, 1111, 1333, 1500, 1759]
    ref = {}
    for c in sample:
        site, ch = divmod(c, cps)
        g0u, g0d = o.build_g0(g0[site, 0]), o.build_g0(g0[site, 1])
        s = o.init_fields(cfg["seed"], site, ch, L)
        Gu, _ = o.dyson(g0u, s, 1, lam)
        Gd, _ = o.dyson(g0d, s, -1, lam)
        ref[c] = dict(site=site, ch=ch, g0u=g0u, g0d=g0d, s=s, Gu=Gu, Gd=Gd, nsw=0, acc=0,
                      bins=np.zeros((nme // bs, 2 * L + 3)))
    o.tie_watch(1e-9)
    done = 0
    while done < nwu + nme:
        w = re if done + re <= nwu else 0
        m = re - w
        hf.hf_sweep(split.handle, w, m, 1 if done == 0 else 0)
        f, cnt = hf.hf_get_fields(split.handle, nc, L)
        assert np.all(cnt == done + re)
        for c, r in ref.items():
            b0 = max(0, done - nwu) // bs
            acc, r["nsw"] = o.run_chain(lam, r["g0u"], r["g0d"], cfg["seed"], r["site"], r["ch"],
                                        r["nsw"], w, m, re, bs, r["s"], r["Gu"], r["Gd"],
                                        r["bins"][b0:])
            r["acc"] += acc
            assert np.array_equal(f[c], r["s"]), "decision mismatch by sweep %d, chain %d" % (done + re, c)
        done += re
    ties = o.tie_count()
    o.tie_watch(0.0)
    print("\nsquare20 whole launch: %d sampled chains x %d proposals, %d near ties (|u - p| < "
          "1e-9 p), decisions identical" % (len(ref), (nwu + nme) * L, ties))
    f2, c2, a2 = _state(hf, split)
    assert np.array_equal(f1, f2) and np.array_equal(c1, c2) and np.array_equal(a1, a2)
    worst_g, worst_b = 0.0, 0.0
    for c, r in ref.items():
        assert a1[c] == r["acc"]
        G1, G2 = hf.hf_get_green(one.handle, c, L), hf.hf_get_green(split.handle, c, L)
        assert np.array_equal(G1, G2)
        worst_g = max(worst_g, _rel(G1[0], r["Gu"]), _rel(G1[1], r["Gd"]))
    assert worst_g < 1e-10, worst_g
    # measured bins: per site, means over chains x bins (the sample's own chains by the oracle)
    for i in sorted({r["site"] for r in ref.values()}):
        g_one = hf.hf_measure(one.handle, i, L)
        g_split = hf.hf_measure(split.handle, i, L)
        assert np.array_equal(g_one[0], g_split[0]) and g_one[2] == g_split[2]
    one.close()
    split.close()


def test_square20_sampled_chain_bins_match_oracle(hf):
    """One site of the 20x20 trap (its 32 chains in one launch of the full 2500 sweeps): the
    site's measured G(tau), n, d, m and their errors against the oracle's 32 chains at 1e-10."""
    cfg = dict(wl.CONFIGS["square20"], precision=0, team_warps=1)
    ctx = hf.Context(hf.make_params(cfg))
    L, ns, cps = ctx.L, ctx.n_sites, cfg["chains_per_site"]
    hf.hf_compute_baths(ctx.handle)
    g0 = hf.hf_get_g0(ctx.handle, ns, L)
    hf.hf_sweep(ctx.handle, cfg["n_warmup"], cfg["n_measure"], 1)
    _, lam = o.constants(cfg["beta"], cfg["U"], L)
    site = 27
    bs, nb = cfg["bin_size"], cfg["n_measure"] // cfg["bin_size"]
    means = []
    for ch in range(cps):
        g0u, g0d = o.build_g0(g0[site, 0]), o.build_g0(g0[site, 1])
        s = o.init_fields(cfg["seed"], site, ch, L)
        Gu, _ = o.dyson(g0u, s, 1, lam)
        Gd, _ = o.dyson(g0d, s, -1, lam)
        bins = np.zeros((nb, 2 * L + 3))
        o.run_chain(lam, g0u, g0d, cfg["seed"], site, ch, 0, cfg["n_warmup"], cfg["n_measure"],
                    cfg["refresh_every"], bs, s, Gu, Gd, bins)
        means.append(bins / bs)
    x = np.concatenate(means)
    mean = x.mean(axis=0)
    err = x.std(axis=0, ddof=1) / np.sqrt(x.shape[0])
    gtau, n, d, m, errs = hf.hf_measure(ctx.handle, site, L)
    assert np.abs(gtau - mean[:2 * L]).max() < 1e-10
    assert abs(n[0] - mean[2 * L]) < 1e-10 and abs(n[1] - mean[2 * L + 1]) < 1e-10
    assert abs(d - mean[2 * L + 2]) < 1e-10
    assert abs(m - (mean[2 * L] - mean[2 * L + 1])) < 1e-10
    assert np.abs(errs[:2 * L + 3] - err).max() < 1e-9
    ctx.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_lambda8_against_brute_force(hf, precision):
    """The 6x6 trap (U = 4, V0 = 0.1, mu = 2, beta = 4) at dtau = 0.5, i.e. L = 8: the CUDA
    sweeps of two impurities (the trap centre and its corner) on the baths of the model's own
    lattice step, against the exact discretised averages over all 2^8 field configurations."""
    cfg = dict(wl.CONFIGS["square6"], dtau=0.5, chains_per_site=512, n_warmup=200,
               n_measure=2000, bin_size=100, max_bins=20, precision=precision, seed=8)
    ctx = hf.Context(hf.make_params(cfg))
    L, ns = ctx.L, ctx.n_sites
    assert L == 8
    hf.hf_compute_baths(ctx.handle)
    g0 = hf.hf_get_g0(ctx.handle, ns, L)
    hf.hf_sweep(ctx.handle, cfg["n_warmup"], cfg["n_measure"], 1)
    rep, _, _ = hf.hf_get_orbits(ctx.handle, ns, 36)
    r2 = [((q % 6) - 2.5) ** 2 + ((q // 6) - 2.5) ** 2 for q in rep]
    _, lam = o.constants(cfg["beta"], cfg["U"], L)
    for site in (int(np.argmin(r2)), int(np.argmax(r2))):
        exact = o.brute_force(lam, o.build_g0(g0[site, 0]), o.build_g0(g0[site, 1]))
        gtau, n, d, m, errs = hf.hf_measure(ctx.handle, site, L)
        z_g = np.abs(gtau.ravel() - exact[:2 * L]) / errs[:2 * L]
        z_n = np.abs(n - exact[2 * L:2 * L + 2]) / errs[2 * L:2 * L + 2]
        z_d = abs(d - exact[2 * L + 2]) / errs[2 * L + 2]
        assert np.all(errs[:2 * L + 3] > 0)
        assert z_n.max() < 3.0 and z_d < 3.0, (site, z_n, z_d)
        assert z_g.max() < 4.0, (site, z_g)
    ctx.close()
