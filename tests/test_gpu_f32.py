"""Mixed-precision path (FP32 sweeps, FP64 Dyson refresh) against the FP64 oracle.

* Deterministic: the FP64 refresh that ends a sweep reproduces the oracle's Dyson recompute for
  the chain's fields (measurement from it within 1e-11, FP32 state within FP32 rounding).
* Statistical: FP32-path observables G(tau), n, d, m agree with the FP64 oracle (and with the
  exact atomic limit) within the combined binned error bars.
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
    cfg = dict(wl.CONFIGS["square6"], precision=1, refresh_every=1)
    cfg.update(over)
    return hf.Context(hf.make_params(cfg)), cfg


@pytest.mark.parametrize("L,dtau", [(16, 0.25), (32, 0.25), (64, 0.25), (128, 0.125)])
def test_refresh_after_fp32_sweeps_matches_oracle_dyson(hf, L, dtau):
    beta = L * dtau
    ctx, cfg = _ctx(hf, chains_per_site=2, beta=beta, dtau=dtau, U=8.0, bin_size=1, max_bins=1,
                    seed=77 + L)
    baths = wl.random_baths(L + 1, ctx.n_sites, beta, L)
    for i in range(ctx.n_sites):
        for sp in range(2):
            hf.hf_set_g0(ctx.handle, i, sp, baths[i, sp])
    hf.hf_sweep(ctx.handle, 6, 1, 1)
    fields, cnt = hf.hf_get_fields(ctx.handle, ctx.n_chains, L)
    assert np.all(cnt == 7)
    acc = hf.hf_get_accepts(ctx.handle, ctx.n_chains)
    assert acc.sum() > 0
    _, lam = o.constants(beta, 8.0, L)
    for i in range(ctx.n_sites):
        g0u, g0d = o.build_g0(baths[i, 0]), o.build_g0(baths[i, 1])
        ref = np.zeros(2 * L + 3)
        for ch in range(2):
            c = 2 * i + ch
            Gu, _ = o.dyson(g0u, fields[c], 1, lam)
            Gd, _ = o.dyson(g0d, fields[c], -1, lam)
            ref += o.measure(Gu, Gd) / 2
            G = hf.hf_get_green(ctx.handle, c, L)
            scale = max(np.abs(Gu).max(), np.abs(Gd).max())
            assert np.abs(G[0] - Gu).max() < 1e-6 * scale
            assert np.abs(G[1] - Gd).max() < 1e-6 * scale
        gtau, n, d, m, errs = hf.hf_measure(ctx.handle, i, L)
        assert np.abs(gtau - ref[:2 * L]).max() < 1e-10
        assert abs(n[0] - ref[2 * L]) < 1e-10 and abs(d - ref[2 * L + 2]) < 1e-10
    ctx.close()


def _gpu_stats(hf, ctx, L, n_warm, n_meas):
    hf.hf_sweep(ctx.handle, n_warm, n_meas, 1)
    out = []
    for i in range(ctx.n_sites):
        gtau, n, d, m, errs = hf.hf_measure(ctx.handle, i, L)
        out.append((np.concatenate([gtau, n, [d]]), errs[:2 * L + 3]))
    return out


def _oracle_stats(L, beta, U, g0u, g0d, chains, n_warm, n_meas, bs, seed, re):
    _, lam = o.constants(beta, U, L)
    xs = []
    for c in range(chains):
        s = o.init_fields(seed, 500, c, L)
        Gu, _ = o.dyson(g0u, s, 1, lam)
        Gd, _ = o.dyson(g0d, s, -1, lam)
        bins = np.zeros((n_meas // bs, 2 * L + 3))
        o.run_chain(lam, g0u, g0d, seed, 500, c, 0, n_warm, n_meas, re, bs, s, Gu, Gd, bins)
        xs.append(bins / bs)
    x = np.concatenate(xs)
    return x.mean(axis=0), x.std(axis=0, ddof=1) / np.sqrt(x.shape[0])


def _z(a, ea, b, eb):
    return np.abs(a - b) / np.sqrt(ea ** 2 + eb ** 2 + 1e-30)


def test_fp32_statistics_match_fp64_oracle_L32(hf):
    L, beta, U, bs, nw, nm = 32, 8.0, 6.0, 100, 200, 3000
    ctx, cfg = _ctx(hf, Lx=1, Ly=1, chains_per_site=16, beta=beta, dtau=0.25, U=U, bin_size=bs,
                    max_bins=nm // bs, seed=11)
    assert ctx.n_sites == 1
    bath = wl.random_baths(31, 1, beta, L)[0]
    hf.hf_set_g0(ctx.handle, 0, 0, bath[0])
    hf.hf_set_g0(ctx.handle, 0, 1, bath[1])
    (mg, eg), = _gpu_stats(hf, ctx, L, nw, nm)
    mo, eo = _oracle_stats(L, beta, U, o.build_g0(bath[0]), o.build_g0(bath[1]), 8, nw, nm, bs,
                           5, 1)
    z = _z(mg, eg, mo, eo)
    assert z.max() < 4.0 and z.mean() < 1.5, (z.max(), z.mean())
    ctx.close()


def test_fp32_atomic_limit_exact(hf):
    # t = 0 single site: Hirsch-Fye is exact; FP32 sweeps must reproduce the closed form.
    # beta = 4 keeps the local moment mobile (at low T whole-chain moment flips are rare and
    # 100-sweep bins would understate the error).
    L, beta, U, eps = 32, 4.0, 4.0, -1.2
    ctx, cfg = _ctx(hf, Lx=1, Ly=1, chains_per_site=16, beta=beta, dtau=0.125, U=U,
                    bin_size=100, max_bins=30, seed=3)
    gt = wl.pole_bath_tau(beta, L, [eps + U / 2], [1.0])
    hf.hf_set_g0(ctx.handle, 0, 0, gt)
    hf.hf_set_g0(ctx.handle, 0, 1, gt)
    (mg, eg), = _gpu_stats(hf, ctx, L, 200, 3000)
    tau = np.arange(L) * beta / L
    Z = 1 + 2 * np.exp(-beta * eps) + np.exp(-beta * (2 * eps + U))
    n = (np.exp(-beta * eps) + np.exp(-beta * (2 * eps + U))) / Z
    dd = np.exp(-beta * (2 * eps + U)) / Z
    g = (np.exp(-eps * tau) + np.exp(-beta * eps) * np.exp(-(eps + U) * tau)) / Z
    exact = np.concatenate([g, g, [n, n, dd]])
    z = np.abs(mg - exact) / (eg + 1e-30)
    assert z.max() < 4.0, z.max()
    ctx.close()


def test_square30_fp32_error_report(hf):
    """The 30x30 trap in the mixed-precision configuration (L = 128, dtau = 0.125, refresh every
    sweep, 16 chains/site): all 1920 chains run on the GPU; one site is replayed by the FP64
    oracle with the same bath; error of G(tau), n and m within the combined error bars."""
    L, bs, nw, nm = 128, 20, 20, 120
    cfg = dict(wl.CONFIGS["square30"], n_warmup=nw, n_measure=nm, bin_size=bs, max_bins=nm // bs)
    ctx = hf.Context(hf.make_params(cfg))
    assert (ctx.n_sites, ctx.n_chains, ctx.L) == (120, 1920, 128)
    baths = wl.random_baths(30, ctx.n_sites, cfg["beta"], L)
    for i in range(ctx.n_sites):
        for sp in range(2):
            hf.hf_set_g0(ctx.handle, i, sp, baths[i, sp])
    stats = _gpu_stats(hf, ctx, L, nw, nm)
    site = 7
    mg, eg = stats[site]
    mo, eo = _oracle_stats(L, cfg["beta"], cfg["U"], o.build_g0(baths[site, 0]),
                           o.build_g0(baths[site, 1]), 6, nw, nm, bs, 9, 1)
    z = _z(mg, eg, mo, eo)
    mz = _z(mg[2 * L] - mg[2 * L + 1], np.hypot(eg[2 * L], eg[2 * L + 1]),
            mo[2 * L] - mo[2 * L + 1], np.hypot(eo[2 * L], eo[2 * L + 1]))
    print("square30 FP32 vs FP64 oracle: max|dG(tau)| = %.2e, |dn| = %.2e, |dm| = %.2e, "
          "max z = %.2f" % (np.abs(mg[:2 * L] - mo[:2 * L]).max(), abs(mg[2 * L] - mo[2 * L]),
                            abs((mg[2 * L] - mg[2 * L + 1]) - (mo[2 * L] - mo[2 * L + 1])), z.max()))
    assert z.max() < 4.5 and mz < 4.0
    ctx.close()
