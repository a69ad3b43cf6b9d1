"""Pins of the oracle's self-consistency iteration (the order of "Model and Methods").

CPU only.  U = 0 makes the impurity problem free, so one iteration must reproduce the free
lattice (numpy eigendecomposition) and a vanishing self-energy; particle-hole symmetry fixes
half filling; the C4v expansion must respect the Hamiltonian.
"""
import numpy as np

from oracle.rdmft import RDMFT


def test_u0_iteration_reproduces_free_lattice():
    r = RDMFT(4, U=0.0, V0=0.2, mu=0.3, beta=3.0, L=12, nw=500, chains=1, h_seed=0.0,
              n_warmup=2, n_measure=20, bin_size=10)
    mean, err = r.iterate()
    assert np.all(err == 0.0)           # G = G0 in every sweep: no variance at all
    lat = r.lat
    e, v = np.linalg.eigh(lat.H0)
    f = 1.0 / (1.0 + np.exp(r.beta * (e - r.mu)))
    nref = (np.abs(v) ** 2 * f[None, :]).sum(axis=1)[r.reps]
    L = r.L
    for sp in range(2):
        assert np.abs(mean[:, 2 * L + sp] - nref).max() < 1e-8
    assert np.abs(r.last["sigma_new"]).max() < 1e-12


def test_seed_and_symmetry_expansion():
    r = RDMFT(6, U=4.0, V0=0.1, mu=2.0, beta=4.0, L=16, nw=8, chains=1, h_seed=0.1)
    full = r.expand_sigma()
    lat = r.lat
    # the seed is U/2 - sigma h eps_i on every site, recovered through the spin-flip map
    for sp, sg in ((0, 1.0), (1, -1.0)):
        assert np.allclose(full[sp, 0, :], 2.0 - sg * 0.1 * lat.parity)
    # a symmetric Sigma-expansion leaves the spin-resolved matrices related by the flips:
    # the static mean-field densities of both spins come out consistent with the orbit map
    for sp in range(2):
        H = lat.H0 + np.diag(full[sp, 0, :].real)
        e, v = np.linalg.eigh(H)
        n = (np.abs(v) ** 2 / (1 + np.exp(4.0 * (e - 2.0)))[None, :]).sum(axis=1)
        other = lat.H0 + np.diag(full[1 - sp, 0, :].real)
        e2, v2 = np.linalg.eigh(other)
        n2 = (np.abs(v2) ** 2 / (1 + np.exp(4.0 * (e2 - 2.0)))[None, :]).sum(axis=1)
        for i in range(lat.N):
            rep = r.reps[r.rep_of[i]]
            src = n2 if r.flip[i] else n
            assert abs(src[rep] - n[i]) < 1e-12


def test_particle_hole_symmetric_lattice_half_filled():
    # V0 = 0, mu = U/2, h = 0 on a bipartite lattice: n = 1 per site (statistical check)
    r = RDMFT(4, U=4.0, V0=0.0, mu=2.0, beta=2.0, L=8, nw=200, chains=4, h_seed=0.0,
              n_warmup=50, n_measure=2000, bin_size=100)
    mean, err = r.iterate()
    L = r.L
    n = mean[:, 2 * L] + mean[:, 2 * L + 1]
    en = np.sqrt(err[:, 2 * L] ** 2 + err[:, 2 * L + 1] ** 2)
    assert np.all(np.abs(n - 1.0) < 4.5 * en + 1e-6)
    # and the bath itself is particle-hole symmetric: g0(tau) = g0(beta - tau)
    g0 = r.last["g0_tau"]
    assert np.abs(g0[:, :, 1:L] - g0[:, :, L - 1:0:-1]).max() < 1e-8
