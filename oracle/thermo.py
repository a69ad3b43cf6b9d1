"""Free-fermion thermodynamics of the one-body lattice H0: the closed forms that pin the entropy
obtained by integrating temperature derivatives of densities ("Results for square lattice":
dS/dmu = dN/dT, integrated from the empty system at mu -> -infinity).

TEST INFRASTRUCTURE ONLY (see the package docstring).

At U = 0 the RDMFT self-consistency is solved by Sigma = 0, and the lattice is a set of
independent levels e_k with orbitals psi_k.  Per spin and level the occupation is
f = 1 / (exp((e_k - mu) / T) + 1) and the entropy is -f ln f - (1 - f) ln(1 - f), so
  N(T, mu)   = 2 sum_k f_k,
  S(T, mu)   = 2 sum_k s(f_k),
  dN/dT      = 2 sum_k f_k (1 - f_k) (e_k - mu) / T^2.
The local forms weight each level by |psi_k(i)|^2: n_i, s_i and dn_i/dT.  For every level,
d s(f)/d mu = d f / d T, so the local entropy s_i is exactly the mu-integral of dn_i/dT from the
empty lattice, the quantity the scan computes site by site; sum_i s_i = S.
"""
from __future__ import annotations

import numpy as np


def _levels(H0):
    e, psi = np.linalg.eigh(H0)
    return e, psi ** 2          # weights w[i, k] = |psi_k(i)|^2


def _fermi(x, T):
    return 0.5 * (1.0 - np.tanh(0.5 * x / T))     # 1 / (e^{x/T} + 1) without overflow


def _two_state_entropy(f):
    out = np.zeros_like(f)
    m = (f > 0.0) & (f < 1.0)
    out[m] = -f[m] * np.log(f[m]) - (1.0 - f[m]) * np.log1p(-f[m])
    return out


def free_density(H0, mu, T):
    """Total density n_i (both spins) of every site."""
    e, w = _levels(H0)
    return w @ (2.0 * _fermi(e - mu, T))


def free_entropy(H0, mu, T):
    """Local entropy s_i of every site (both spins); their sum is the total entropy S."""
    e, w = _levels(H0)
    return w @ (2.0 * _two_state_entropy(_fermi(e - mu, T)))


def free_dndT(H0, mu, T):
    """Temperature derivative of n_i at fixed mu (both spins)."""
    e, w = _levels(H0)
    f = _fermi(e - mu, T)
    return w @ (2.0 * f * (1.0 - f) * (e - mu) / T ** 2)
