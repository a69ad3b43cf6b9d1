"""Parity of the lattice step (eq. 2) and of whole RDMFT iterations on the three-dimensional
lattices ("Efficient simulations for three dimensions": trapped boxes with periodic boundaries and
slabs periodic across their layers), through the C ABI, with the CPU oracle.

Cases span both forms of the lattice step -- the band L D L^T and selected inversion in a
shared-memory window (one warp per matrix for band half-width b <= 32, one block above; taken
below b = 128, or when asked for with lattice_form = 2), and the blocked band L D L^T in global
memory with forward solves at one site per orbit and spin (taken from b = 128 on, its products
on the tensor cores up to b = 520, or when asked for with lattice_form = 1) -- and both spin
treatments (spin-down matrices inverted, or read from the spin-up ones through a
sublattice-exchanging symmetry).  The
periodic 14^3 and 16^3 boxes of Fig. 4 (b = 392, 512) run in the blocked form.  Bars as for the square: G_ii(i w_n) within 1e-12
relative; baths within 1e-12; decisions identical; observables within 1e-10; Sigma within 1e-9
relative.
"""
import numpy as np
import pytest

from oracle.lattice import lattice_entries, lattice_step
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


def _cfg(geom, Lx, Ly, Lz, per, **over):
    d = dict(wl.CONFIGS["square6"], geometry=geom, Lx=Lx, Ly=Ly, Lz=Lz, periodic=per, V0=0.07,
             mu=1.1, n_matsubara=40, chains_per_site=1, n_warmup=1, n_measure=2, bin_size=1,
             max_bins=2)
    d.update(over)
    return d


def _causal_sigma(rng, ns, nw, beta, U):
    wn = (2 * np.arange(nw) + 1) * np.pi / beta
    return (U / 2 + rng.uniform(-0.5, 0.5, (ns, 2, 1))
            - 1j * rng.uniform(0.05, 0.6, (ns, 2, 1)) / (1.0 + wn[None, None, :]))


# geometry, Lx, Ly, Lz, periodic, band half-width, spin-halved
SMALL = [
    (2, 4, 4, 4, 1, 32, True),      # narrow kernel
    (2, 5, 5, 5, 0, 25, False),     # narrow, odd box: no sublattice exchange
    (3, 6, 6, 4, 0, 24, True),      # narrow slab
    (2, 6, 6, 6, 0, 36, True),      # wide kernel
    (2, 7, 7, 7, 0, 49, False),     # wide, both spins inverted
    (3, 8, 6, 4, 1, 64, True),      # wide, periodic slab
    (0, 20, 20, 1, 1, 40, True),    # periodic square: folded band
]


@pytest.mark.parametrize("form", [2, 1])   # the window form, the blocked form
@pytest.mark.parametrize("geom,Lx,Ly,Lz,per,band,halved",
                         SMALL + [(0, 6, 6, 1, 0, 6, True),     # b < panel width (blocked form)
                                  (2, 8, 8, 8, 1, 128, True)])  # b = 128: the blocked form's
                                                                # products on the tensor cores
def test_lattice_step_all_frequencies(hf, geom, Lx, Ly, Lz, per, band, halved, form):
    """Every inequivalent site and every frequency of a set self-energy against a dense
    inverse, in either form of the lattice step."""
    cfg = _cfg(geom, Lx, Ly, Lz, per, lattice_form=form)
    p = hf.make_params(cfg)
    N, ns, b, nsp, _, _, _ = hf.hf_lattice_info(p)
    assert b == band
    ctx = hf.Context(p)
    assert hf.hf_get_lattice_plan(ctx.handle)[0] == (1 if form == 1 else 0)
    ref = _oracle_for(cfg)
    assert ns == ref.nsite and N == ref.lat.N
    has_flip = any(np.all(ref.lat.parity[im] != ref.lat.parity) for im in ref.lat._images)
    assert has_flip == halved and nsp == (1 if halved else 2)
    rng = np.random.default_rng(geom * 100 + Lx)
    sig = _causal_sigma(rng, ns, ctx.nw, cfg["beta"], cfg["U"])
    hf.hf_set_sigma(ctx.handle, sig)
    hf.hf_compute_baths(ctx.handle)
    gloc = hf.hf_get_gloc(ctx.handle, ns, ctx.nw)
    ref.sigma = sig.copy()
    full = ref.expand_sigma()
    for sp in range(2):
        want = lattice_step(ref.lat.H0, cfg["mu"], cfg["beta"], full[sp])[:, ref.reps]
        assert np.abs(gloc[:, sp, :].T - want).max() < 1e-12 * np.abs(want).max(), sp
    # the baths built from it (Weiss field, tails with six neighbours, i w -> tau)
    _, gw_t = ref.weiss(np.transpose(np.array([
        lattice_step(ref.lat.H0, cfg["mu"], cfg["beta"], full[sp])[:, ref.reps] for sp in range(2)]),
        (2, 0, 1)))
    want_tau = ref.bath_tau(gw_t)[:, :, :ctx.L]
    assert np.abs(hf.hf_get_g0(ctx.handle, ns, ctx.L) - want_tau).max() < 1e-12
    ctx.close()


LARGE = [
    (3, 24, 24, 4, 0, 96, 0),       # slab of 2304 sites (window form)
    (2, 8, 8, 8, 1, 128, 2),        # periodic box of 512 sites, in the window form
    (2, 12, 12, 12, 0, 144, 2),     # open box of 1728 sites, in the window form
    (2, 12, 12, 12, 0, 144, 0),     # the same in the form taken by default (blocked band form)
    (2, 14, 14, 14, 1, 392, 0),     # periodic boxes of Fig. 4 (blocked band form)
    (2, 16, 16, 16, 1, 512, 0),
]


@pytest.mark.parametrize("geom,Lx,Ly,Lz,per,band,form", LARGE)
def test_lattice_step_large_sampled(hf, geom, Lx, Ly, Lz, per, band, form):
    """Full-size lattices at 500 frequencies: sampled (frequency, spin, orbit) entries against one
    oracle column of M^{-1} each (sparse LU); every orbit for the blocked band form."""
    cfg = _cfg(geom, Lx, Ly, Lz, per, V0=0.03, mu=2.0, U=8.0, beta=8.0, dtau=0.25,
               n_matsubara=500, n_measure=1, max_bins=1, lattice_form=form)
    p = hf.make_params(cfg)
    _, ns, b, _, _, _, _ = hf.hf_lattice_info(p)
    assert b == band
    ctx = hf.Context(p)
    wide = hf.hf_get_lattice_plan(ctx.handle)[0]
    assert wide == (1 if (form == 1 or (form == 0 and band >= 128) or band > 165) else 0)
    hf.hf_compute_baths(ctx.handle)          # lattice step from the seeded self-energy
    gloc = hf.hf_get_gloc(ctx.handle, ns, ctx.nw)
    ref = _oracle_for(cfg)
    full = ref.expand_sigma()
    orbits = list(range(ns)) if wide else sorted({0, 1, ns // 2, ns - 1})
    sites = [int(ref.reps[o]) for o in orbits]
    for n in (0, 7, 250, 499):
        for sp in range(2):
            want = lattice_entries(ref.lat.H0, cfg["mu"], cfg["beta"], full[sp][n], n, sites)
            got = gloc[orbits, sp, n]
            assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), (n, sp)
    ctx.close()


@pytest.mark.parametrize("precision,form", [(0, 0), (2, 0), (0, 1)])
def test_rdmft_iteration_periodic_box_full(hf, precision, form):
    """4x4x4 periodic trapped box (4 inequivalent sites), U = 4, beta = 4, L = 16, 500 + 2000
    sweeps: two complete iterations compared step by step with the oracle (form 1: the lattice
    step in the blocked band form)."""
    cfg = dict(wl.CONFIGS["square6"], geometry=2, Lx=4, Ly=4, Lz=4, periodic=1, V0=0.15, mu=2.0,
               precision=precision, lattice_form=form)
    ctx = hf.Context(hf.make_params(cfg))
    ref = _oracle_for(cfg)
    assert ctx.n_sites == 4
    L, ns, nw = ctx.L, ctx.n_sites, ctx.nw
    for it in range(2):
        hf.hf_rdmft_step(ctx.handle)
        mean, err = ref.iterate()
        gloc = hf.hf_get_gloc(ctx.handle, ns, nw)
        assert np.abs(gloc - ref.last["Gloc"]).max() < 1e-12 * np.abs(ref.last["Gloc"]).max()
        g0 = hf.hf_get_g0(ctx.handle, ns, L)
        assert np.abs(g0 - ref.last["g0_tau"][:, :, :L]).max() < 1e-12
        f, cnt = hf.hf_get_fields(ctx.handle, ctx.n_chains, L)
        assert np.array_equal(f, ref.fields.reshape(ctx.n_chains, L)), "iteration %d" % it
        m_gpu, e_gpu = hf.hf_get_observables(ctx.handle, ns, L)
        assert np.abs(m_gpu[:, :2 * L + 3] - mean).max() < 1e-10
        assert np.abs(e_gpu[:, :2 * L + 3] - err).max() < 1e-10
        sig = hf.hf_get_sigma(ctx.handle, ns, nw)
        assert np.abs(sig - ref.sigma).max() < 1e-9 * np.abs(ref.sigma).max()
    ctx.close()
