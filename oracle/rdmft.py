"""One real-space DMFT self-consistency iteration, in the order of the paper.

TEST INFRASTRUCTURE ONLY (see the package docstring).

"Model and Methods": eq. 2 couples G and Sigma only at equal Matsubara frequency (lattice step,
independent per frequency); the impurity problems, one per inequivalent site, are solved by
Hirsch-Fye QMC at fixed dtau.  Readings used where the paper is silent (each one also stated in
the design notes): Hartree-shifted bath 1/G~0 = 1/G0 - U/2 for the symmetric decoupling;
iteration 0 seeds Sigma_{i sigma} = U/2 - sigma h eps_i (eps_i = sublattice parity); linear
mixing Sigma <- mix Sigma_new + (1 - mix) Sigma_old; chains keep their Ising fields across
iterations (warm start) and re-anchor G by a Dyson refresh from the new bath.
"""
from __future__ import annotations

import numpy as np

from . import core
from .fourier import iw_to_tau, tau_to_iw
from .lattice import Lattice, lattice_step


class RDMFT:
    def __init__(self, Lx, Ly=None, geometry=0, periodic=False, t=1.0, U=4.0, V0=0.1, mu=2.0,
                 beta=4.0, L=16, nw=500, chains=1, seed=1, h_seed=0.1, mix=0.5,
                 n_warmup=500, n_measure=2000, refresh_every=10, bin_size=100, refresh_stagger=0,
                 Lz=1):
        self.lat = Lattice(Lx, Ly, geometry=geometry, periodic=periodic, t=t, V0=V0, Lz=Lz)
        self.reps, self.rep_of, self.flip = self.lat.orbits()
        self.U, self.mu, self.beta, self.L, self.nw = U, mu, beta, L, nw
        self.t = t
        self.chains, self.seed, self.mix = chains, seed, mix
        self.n_warmup, self.n_measure = n_warmup, n_measure
        self.refresh_every, self.bin_size = refresh_every, bin_size
        self.refresh_stagger = refresh_stagger
        self.dtau, self.lam = core.constants(beta, U, L)
        ns = len(self.reps)
        self.nsite = ns
        eps = self.lat.parity[self.reps]
        self.sigma = np.zeros((ns, 2, nw), dtype=np.complex128)
        for sp, sg in ((0, 1.0), (1, -1.0)):
            self.sigma[:, sp, :] = (U / 2.0 - sg * h_seed * eps)[:, None]
        self.fields = np.zeros((ns, chains, L), dtype=np.int8)
        for i in range(ns):
            for c in range(chains):
                self.fields[i, c] = core.init_fields(seed, i, c, L)
        self.nsw = np.zeros((ns, chains), dtype=np.uint32)
        self.accepts = np.zeros((ns, chains), dtype=np.int64)

    # -- pieces ----------------------------------------------------------
    def expand_sigma(self):
        """Sigma on all N sites: Sigma_{i, sigma} = Sigma_{rep(i), sigma xor flip(i)}. [2, nw, N]"""
        N = self.lat.N
        full = np.zeros((2, self.nw, N), dtype=np.complex128)
        for i in range(N):
            for sp in range(2):
                full[sp, :, i] = self.sigma[self.rep_of[i], sp ^ int(self.flip[i]), :]
        return full

    def weiss(self, Gloc_rep):
        """Bath of each impurity: 1/G0 = 1/G_ii + Sigma_i, shifted 1/G~0 = 1/G0 - U/2."""
        weiss_inv = 1.0 / Gloc_rep + self.sigma
        gw_t = 1.0 / (weiss_inv - self.U / 2.0)
        return weiss_inv, gw_t

    def tails(self):
        """High-frequency coefficients of G~0: c2 = V_i - mu + U/2, c3 = c2^2 + z_i t^2."""
        V = self.lat.V[self.reps]
        z = self.lat.z[self.reps]
        c2 = V - self.mu + self.U / 2.0
        c3 = c2 ** 2 + z * self.t ** 2
        return c2, c3

    def bath_tau(self, gw_t):
        c2, c3 = self.tails()
        out = np.zeros((self.nsite, 2, self.L + 1))
        for i in range(self.nsite):
            for sp in range(2):
                out[i, sp] = iw_to_tau(self.beta, gw_t[i, sp], c2[i], c3[i], self.L)
        return out

    def impurities(self, g0_tau):
        """Warm-started QMC of every chain; returns per-chain bins [ns, chains, nbins, 2L+3]."""
        L = self.L
        nb = self.n_measure // self.bin_size
        bins = np.zeros((self.nsite, self.chains, nb, 2 * L + 3))
        self.G_last = np.zeros((self.nsite, self.chains, 2, L, L))
        for i in range(self.nsite):
            g0up = core.build_g0(g0_tau[i, 0, :L])
            g0dn = core.build_g0(g0_tau[i, 1, :L])
            for c in range(self.chains):
                s = self.fields[i, c]
                Gup, _ = core.dyson(g0up, s, +1, self.lam)
                Gdn, _ = core.dyson(g0dn, s, -1, self.lam)
                acc, nsw = core.run_chain(self.lam, g0up, g0dn, self.seed, i, c,
                                          int(self.nsw[i, c]), self.n_warmup, self.n_measure,
                                          self.refresh_every, self.bin_size, s, Gup, Gdn,
                                          bins[i, c], refresh_stagger=self.refresh_stagger)
                self.nsw[i, c] = nsw
                self.accepts[i, c] += acc
                self.G_last[i, c, 0] = Gup
                self.G_last[i, c, 1] = Gdn
        return bins

    def reduce(self, bins):
        """Mean over chains and bins, error = std / sqrt(#samples) of the bin averages."""
        x = bins / float(self.bin_size)
        ns = x.shape[0]
        x = x.reshape(ns, -1, x.shape[-1])
        mean = x.mean(axis=1)
        cnt = x.shape[1]
        err = x.std(axis=1, ddof=1) / np.sqrt(cnt) if cnt > 1 else np.zeros_like(mean)
        return mean, err

    # -- one iteration -----------------------------------------------------
    def iterate(self):
        L = self.L
        full = self.expand_sigma()
        Gloc = np.zeros((self.nsite, 2, self.nw), dtype=np.complex128)
        for sp in range(2):
            g = lattice_step(self.lat.H0, self.mu, self.beta, full[sp])
            Gloc[:, sp, :] = g[:, self.reps].T
        weiss_inv, gw_t = self.weiss(Gloc)
        g0_tau = self.bath_tau(gw_t)
        bins = self.impurities(g0_tau)
        mean, err = self.reduce(bins)
        gimp = np.zeros((self.nsite, 2, self.nw), dtype=np.complex128)
        for i in range(self.nsite):
            for sp in range(2):
                gimp[i, sp] = tau_to_iw(self.beta, mean[i, sp * L:(sp + 1) * L],
                                        g0_tau[i, sp, :L], gw_t[i, sp])
        sigma_new = weiss_inv - 1.0 / gimp
        self.sigma = self.mix * sigma_new + (1.0 - self.mix) * self.sigma
        self.last = dict(Gloc=Gloc, weiss_inv=weiss_inv, gw_t=gw_t, g0_tau=g0_tau, bins=bins,
                         mean=mean, err=err, gimp=gimp, sigma_new=sigma_new)
        return mean, err
