"""Parity of the CUDA RDMFT iteration (lattice step, transforms, impurities, self-energy)
with the CPU oracle, through the C ABI.

Bars: orbit tables bit-exact; lattice step G_ii(i w_n) within 1e-12 relative; bath g~0(tau)
within 1e-12; impurity decisions identical; observables within 1e-10; self-energy within 1e-9
relative over a whole iteration (1/G_imp ~ i w_n at high frequency, so the observables' 1e-10
grows by |w_n| / |Sigma|).  The frequency-domain steps alone, fed the GPU's own inputs (the
Weiss field, the tau -> i w_n spline transform of the measured G(tau), the unmixed and the mixed
self-energy), are held to 1e-12.
"""
import numpy as np
import pytest

from oracle.fourier import tau_to_iw
from oracle.lattice import Lattice, lattice_entries, lattice_step
from oracle.rdmft import RDMFT
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


def _oracle_for(cfg):
    L = int(round(cfg["beta"] / cfg["dtau"]))
    return RDMFT(cfg["Lx"], cfg.get("Ly"), geometry=cfg.get("geometry", 0),
                 periodic=bool(cfg.get("periodic", 0)), t=cfg.get("t", 1.0), U=cfg["U"],
                 V0=cfg["V0"], mu=cfg["mu"], beta=cfg["beta"], L=L, nw=cfg["n_matsubara"],
                 chains=cfg["chains_per_site"], seed=cfg["seed"], h_seed=cfg["h_seed"],
                 mix=cfg["mix"], n_warmup=cfg["n_warmup"], n_measure=cfg["n_measure"],
                 refresh_every=cfg["refresh_every"], bin_size=cfg["bin_size"],
                 refresh_stagger=cfg.get("refresh_stagger", 0), Lz=cfg.get("Lz", 1))


@pytest.mark.parametrize("Lx,geom", [(6, 0), (20, 0), (30, 0), (40, 1), (7, 1)])
def test_orbit_tables_bit_exact(hf, Lx, geom):
    cfg = dict(wl.CONFIGS["square6"], Lx=Lx, Ly=Lx, geometry=geom, n_matsubara=4,
               chains_per_site=1)
    p = hf.make_params(cfg)
    # sizes and orbit tables are host-side: a tiny context is enough
    ctx = hf.Context(p)
    rep, rep_of, flip = hf.hf_get_orbits(ctx.handle, ctx.n_sites, ctx.N)
    lat = Lattice(Lx, Lx if geom == 0 else None, geometry=geom)
    r2, ro2, f2 = lat.orbits()
    assert np.array_equal(rep, r2) and np.array_equal(rep_of, ro2) and np.array_equal(flip, f2)
    ctx.close()


@pytest.mark.parametrize("precision", [0, 2])
def test_rdmft_iteration_square6_full(hf, precision):
    """The 6x6 trap (U=4, V0=0.1, mu=2, beta=4, L=16), 1 chain/site, 500 + 2000 sweeps: two
    complete iterations, each compared step by step with the oracle (FP64 and FP32-pair
    sweeps)."""
    cfg = dict(wl.CONFIGS["square6"], precision=precision)
    ctx = hf.Context(hf.make_params(cfg))
    ref = _oracle_for(cfg)
    L, ns, nw = ctx.L, ctx.n_sites, ctx.nw
    for it in range(2):
        hf.hf_rdmft_step(ctx.handle)
        mean, err = ref.iterate()
        gloc = hf.hf_get_gloc(ctx.handle, ns, nw)
        g0 = hf.hf_get_g0(ctx.handle, ns, L)
        assert np.abs(gloc - ref.last["Gloc"]).max() < 1e-12 * np.abs(ref.last["Gloc"]).max()
        assert np.abs(g0 - ref.last["g0_tau"][:, :, :L]).max() < 1e-12
        f, cnt = hf.hf_get_fields(ctx.handle, ctx.n_chains, L)
        assert np.array_equal(f, ref.fields.reshape(ctx.n_chains, L)), "iteration %d" % it
        assert np.all(cnt == (it + 1) * 2500)
        m_gpu, e_gpu = hf.hf_get_observables(ctx.handle, ns, L)
        assert np.abs(m_gpu[:, :2 * L + 3] - mean).max() < 1e-10
        assert np.abs(e_gpu[:, :2 * L + 3] - err).max() < 1e-10
        sig = hf.hf_get_sigma(ctx.handle, ns, nw)
        assert np.abs(sig - ref.sigma).max() < 1e-9 * np.abs(ref.sigma).max()
    ctx.close()


def _rel(got, want):
    return np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("precision", [0, 2])
def test_frequency_steps_on_the_gpus_own_inputs(hf, precision):
    """The 6x6 trap, two iterations: each frequency-domain step against the oracle's definition
    applied to the GPU's own inputs, so that the QMC's 1e-10 agreement does not enter.  Weiss
    field 1/G0 = 1/G_ii + Sigma and G~0 = 1/(1/G0 - U/2) from the GPU's G_ii and Sigma; the
    impurity G(i w_n) = G~0 + FT[-spline(g_imp - g~0)] from the GPU's measured G(tau), bath
    g~0(tau) and G~0(i w_n) (oracle.fourier.tau_to_iw); Sigma_new = 1/G0 - 1/G_imp; the mixed
    Sigma = mix Sigma_new + (1 - mix) Sigma_old."""
    cfg = dict(wl.CONFIGS["square6"], precision=precision)
    ctx = hf.Context(hf.make_params(cfg))
    ref = _oracle_for(cfg)
    L, ns, nw, beta, mix = ctx.L, ctx.n_sites, ctx.nw, cfg["beta"], cfg["mix"]
    for it in range(2):
        sig_old = hf.hf_get_sigma(ctx.handle, ns, nw)
        hf.hf_rdmft_step(ctx.handle)
        gloc = hf.hf_get_gloc(ctx.handle, ns, nw)
        g0 = hf.hf_get_g0(ctx.handle, ns, L)
        mean, _ = hf.hf_get_observables(ctx.handle, ns, L)
        gw0, winv, gimp, snew = hf.hf_get_impurity_iw(ctx.handle, ns, nw)
        ref.sigma = sig_old.copy()
        w_ref, gw_ref = ref.weiss(gloc)
        assert _rel(winv, w_ref) < 1e-12, it
        assert _rel(gw0, gw_ref) < 1e-12, it
        want = np.zeros_like(gimp)
        for i in range(ns):
            for sp in range(2):
                want[i, sp] = tau_to_iw(beta, mean[i, sp * L:(sp + 1) * L], g0[i, sp], gw0[i, sp])
        assert _rel(gimp, want) < 1e-12, (it, _rel(gimp, want))
        assert _rel(snew, winv - 1.0 / gimp) < 1e-12, it
        sig = hf.hf_get_sigma(ctx.handle, ns, nw)
        assert _rel(sig, mix * snew + (1.0 - mix) * sig_old) < 1e-14, it
    ctx.close()


def test_lattice_step_square20_sampled_frequencies(hf):
    """The 20x20 trap (N = 400, band half-width 20): one iteration's lattice step from the
    seeded self-energy, every site of the sampled frequencies against a dense inverse."""
    cfg = dict(wl.CONFIGS["square20"], chains_per_site=1, n_warmup=1, n_measure=2, bin_size=1,
               max_bins=2)
    ctx = hf.Context(hf.make_params(cfg))
    hf.hf_rdmft_step(ctx.handle)
    gloc = hf.hf_get_gloc(ctx.handle, ctx.n_sites, ctx.nw)
    ref = _oracle_for(cfg)
    full = ref.expand_sigma()
    idx = np.array([0, 1, 57, 250, 499])
    for sp in range(2):
        g = lattice_step(ref.lat.H0, cfg["mu"], cfg["beta"], full[sp][idx], n_index=idx)
        want = g[:, ref.reps]
        got = gloc[:, sp, idx].T
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    ctx.close()


def test_lattice_step_disc_all_frequencies(hf):
    """Site-centred disc (radius 6, N = 113): band from the row numbering of a disc."""
    cfg = dict(wl.CONFIGS["square6"], Lx=6, geometry=1, V0=0.08, mu=1.0, n_matsubara=40,
               chains_per_site=1, n_warmup=1, n_measure=2, bin_size=1, max_bins=2)
    ctx = hf.Context(hf.make_params(cfg))
    hf.hf_rdmft_step(ctx.handle)
    gloc = hf.hf_get_gloc(ctx.handle, ctx.n_sites, ctx.nw)
    ref = _oracle_for(cfg)
    full = ref.expand_sigma()
    for sp in range(2):
        want = lattice_step(ref.lat.H0, cfg["mu"], cfg["beta"], full[sp])[:, ref.reps]
        assert np.abs(gloc[:, sp, :].T - want).max() < 1e-12 * np.abs(want).max()
    ctx.close()


@pytest.mark.parametrize("geom,Lx", [(0, 6), (1, 6)])
def test_compute_baths_from_a_set_self_energy(hf, geom, Lx):
    """hf_set_sigma + hf_compute_baths (lattice step, Weiss fields, iw -> tau with tails) against
    the oracle's steps, for an arbitrary causal self-energy (Im Sigma <= 0 on w_n > 0)."""
    cfg = dict(wl.CONFIGS["square6"], Lx=Lx, Ly=Lx, geometry=geom, V0=0.08, mu=1.3,
               n_matsubara=64, chains_per_site=1, n_warmup=1, n_measure=2, bin_size=1, max_bins=2)
    ctx = hf.Context(hf.make_params(cfg))
    ns, nw, L = ctx.n_sites, ctx.nw, ctx.L
    rng = np.random.default_rng(7 + geom)
    wn = (2 * np.arange(nw) + 1) * np.pi / cfg["beta"]
    sig = (cfg["U"] / 2 + rng.uniform(-0.5, 0.5, (ns, 2, 1))
           - 1j * rng.uniform(0.05, 0.6, (ns, 2, 1)) / (1.0 + wn[None, None, :]))
    hf.hf_set_sigma(ctx.handle, sig)
    hf.hf_compute_baths(ctx.handle)
    ref = _oracle_for(cfg)
    ref.sigma = sig.copy()
    full = ref.expand_sigma()
    Gloc = np.zeros((ns, 2, nw), dtype=np.complex128)
    for sp in range(2):
        Gloc[:, sp, :] = lattice_step(ref.lat.H0, cfg["mu"], cfg["beta"], full[sp])[:, ref.reps].T
    _, gw_t = ref.weiss(Gloc)
    want = ref.bath_tau(gw_t)[:, :, :L]
    assert np.abs(hf.hf_get_gloc(ctx.handle, ns, nw) - Gloc).max() < 1e-12 * np.abs(Gloc).max()
    assert np.abs(hf.hf_get_g0(ctx.handle, ns, L) - want).max() < 1e-12
    ctx.close()


def test_lattice_step_disc40_full_size_sampled(hf):
    """The largest lattice in use (site-centred disc of radius 40: N = 5025, 663 inequivalent
    sites) at the serving workload's parameters: the GPU band solver against one oracle column of
    M^{-1} per sampled (frequency, spin, site), from the seeded self-energy."""
    cfg = dict(wl.CONFIGS["square6"], Lx=40, Ly=40, geometry=1, U=8.0, V0=0.010, mu=4.0,
               beta=8.0, dtau=0.25, n_matsubara=500, chains_per_site=1, n_warmup=1, n_measure=1,
               bin_size=1, max_bins=1)
    ctx = hf.Context(hf.make_params(cfg))
    assert ctx.n_sites == 663
    hf.hf_compute_baths(ctx.handle)
    gloc = hf.hf_get_gloc(ctx.handle, ctx.n_sites, ctx.nw)
    ref = _oracle_for(cfg)
    assert ref.lat.N == 5025
    full = ref.expand_sigma()
    orbits = [0, 1, 331, 662]
    sites = [int(ref.reps[o]) for o in orbits]
    for n in (0, 1, 123, 499):
        for sp in range(2):
            want = lattice_entries(ref.lat.H0, cfg["mu"], cfg["beta"], full[sp][n], n, sites)
            got = gloc[orbits, sp, n]
            assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), (n, sp)
    ctx.close()
