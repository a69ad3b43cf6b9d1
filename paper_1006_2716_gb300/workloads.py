"""Synthetic workloads: the trapped-lattice configurations and seeded input generators.

This module holds parameters and seeded random inputs only -- none of the solver's arithmetic.
It is the one module that both the tests of the CUDA path and the oracle-side tests draw their
inputs from, so that both sides see identical bytes.

Configurations (the trapped 2D Hubbard model of eq. 1 with V_i = V0 r_i^2, t = 1):

* ``square6``   -- 6x6 open square, U=4, V0=0.1, mu=2, beta=4, dtau=0.25 (L=16), 1 chain per
  inequivalent site, 500 + 2000 sweeps, staggered seed field h=0.1, seed 1.
* ``square20``  -- 20x20 open square, U=8, V0=0.05, beta=8, dtau=0.25 (L=32), 32 chains per site
  (55 sites -> 1760 chains), mu fixed so that the seeded mean-field cloud holds ~100 atoms.
* ``scan20``    -- the square20 trap at beta in {5, 8, 10, 16} (L = 20, 32, 40, 64), batched.
* ``square30``  -- 30x30 open square, U=8, V0=0.03, beta=16, dtau=0.125 (L=128), 16 chains per
  site (120 sites), single-precision sweeps with a double-precision refresh every sweep.
* ``disc40``    -- site-centred disc of radius 40 (5025 sites, 663 inequivalent), U=8; impurity
  solve requests at L in {32, 40, 64}.
* ``slab16``    -- three dimensions, the reduced system of "Efficient simulations for three
  dimensions": a 16x16 slab of 4 layers, periodic in all three directions, cylindrical trap
  V0=0.05, U=8, mu=4 (half filling at the axis), T = 0.41 (beta=2.4), dtau=0.1 (L=24), 32 chains
  per inequivalent site (36 sites).
* ``box12``     -- a 12x12x12 open box with a spherical trap V0=0.08, otherwise as slab16
  (56 inequivalent sites).
* ``box14p``, ``box16p`` -- the periodic cubic boxes of Fig. 4: 14^3 and 16^3 sites, periodic in
  all three directions (band half-width 392 and 512 in the folded band order), spherical trap
  V0=0.05, U=12, T = 0.33 (beta=3), mu = U/2 (half filling at the centre; the figure does not
  state mu), dtau=0.125 (L=24), 16 chains per inequivalent site (84 and 120 sites).
"""
from __future__ import annotations

import numpy as np

# chemical potentials fixed once so that the seeded static mean field (Sigma = U/2 -+ h eps_i)
# holds 100 atoms (square20, beta = 8) and 200 atoms (square30, beta = 16)
MU_SQUARE20 = 3.9527

CONFIGS = {
    "square6": dict(Lx=6, Ly=6, geometry=0, periodic=0, t=1.0, U=4.0, V0=0.1, mu=2.0, beta=4.0,
                    dtau=0.25, n_matsubara=500, chains_per_site=1, n_warmup=500, n_measure=2000,
                    refresh_every=10, bin_size=100, seed=1, h_seed=0.1, mix=0.5),
    "square20": dict(Lx=20, Ly=20, geometry=0, periodic=0, t=1.0, U=8.0, V0=0.05,
                     mu=MU_SQUARE20, beta=8.0, dtau=0.25, n_matsubara=500, chains_per_site=32,
                     n_warmup=500, n_measure=2000, refresh_every=10, bin_size=100, seed=2,
                     h_seed=0.1, mix=0.5),
    "square30": dict(Lx=30, Ly=30, geometry=0, periodic=0, t=1.0, U=8.0, V0=0.03, mu=4.2571,
                     beta=16.0, dtau=0.125, precision=1, n_matsubara=500, chains_per_site=16,
                     n_warmup=500,
                     n_measure=2000, refresh_every=1, bin_size=100, seed=4, h_seed=0.1,
                     mix=0.5),
    "slab16": dict(Lx=16, Ly=16, Lz=4, geometry=3, periodic=1, t=1.0, U=8.0, V0=0.05, mu=4.0,
                   beta=2.4, dtau=0.1, precision=2, team_warps=1, n_matsubara=500,
                   chains_per_site=32, n_warmup=500, n_measure=2000, refresh_every=10,
                   bin_size=100, seed=5, h_seed=0.1, mix=0.5),
    "box14p": dict(Lx=14, Ly=14, Lz=14, geometry=2, periodic=1, t=1.0, U=12.0, V0=0.05, mu=6.0,
                   beta=3.0, dtau=0.125, precision=2, team_warps=1, n_matsubara=500,
                   chains_per_site=16, n_warmup=500, n_measure=2000, refresh_every=10,
                   bin_size=100, seed=7, h_seed=0.1, mix=0.5),
    "box16p": dict(Lx=16, Ly=16, Lz=16, geometry=2, periodic=1, t=1.0, U=12.0, V0=0.05, mu=6.0,
                   beta=3.0, dtau=0.125, precision=2, team_warps=1, n_matsubara=500,
                   chains_per_site=16, n_warmup=500, n_measure=2000, refresh_every=10,
                   bin_size=100, seed=8, h_seed=0.1, mix=0.5),
    "box12": dict(Lx=12, Ly=12, Lz=12, geometry=2, periodic=0, t=1.0, U=8.0, V0=0.08, mu=4.0,
                  beta=2.4, dtau=0.1, precision=2, team_warps=1, n_matsubara=500,
                  chains_per_site=32, n_warmup=500, n_measure=2000, refresh_every=10,
                  bin_size=100, seed=6, h_seed=0.1, mix=0.5),
}
SCAN20_BETAS = (5.0, 8.0, 10.0, 16.0)


def bath_poles(seed: int, n_poles: int = 4, spread: float = 2.5, shift: float = 0.0):
    """Random discrete bath: pole energies in [-spread, spread] + shift, positive weights
    summing to one (a valid non-interacting spectral function)."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(-spread, spread, n_poles) + shift
    w = rng.uniform(0.2, 1.0, n_poles)
    return e, w / w.sum()


def pole_bath_tau(beta: float, L: int, e, w):
    """Positive-convention free Green function sum_k w_k e^{-e_k tau}/(1 + e^{-beta e_k}) at
    tau_m = m beta / L, m = 0..L-1 (tau_0 = 0+): the input bath of one impurity."""
    tau = np.arange(L) * (beta / L)
    e = np.asarray(e, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros(L)
    for ek, wk in zip(e, w):
        if ek >= 0:
            out += wk * np.exp(-ek * tau) / (1.0 + np.exp(-beta * ek))
        else:  # same value, written without overflow for negative energies
            out += wk * np.exp(ek * (beta - tau)) / (np.exp(beta * ek) + 1.0)
    return out


def random_baths(seed: int, n: int, beta: float, L: int, n_poles: int = 4):
    """[n, 2, L] baths (spin up / down differ, as in an ordered phase) for n impurities."""
    out = np.zeros((n, 2, L))
    for i in range(n):
        for sp in range(2):
            e, w = bath_poles(seed * 1000003 + 2 * i + sp, n_poles,
                              shift=(0.3 if sp == 0 else -0.3))
            out[i, sp] = pole_bath_tau(beta, L, e, w)
    return out
