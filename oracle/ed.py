"""Exact diagonalisation of a small Anderson impurity: the continuous-time answer (dtau -> 0) that
the Hirsch-Fye discretisation approaches.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The impurity problem of "Model and Methods" with a bath given by poles: the Hartree-shifted free
impurity Green function g~0(tau) = sum_k w_k e^{-e_k tau} / (1 + e^{-beta e_k}) (weights w_k > 0,
sum 1) is the impurity element of a single-particle Hamiltonian h = V diag(e) V^T whose orthogonal
V has first row sqrt(w).  The interacting impurity adds, in the split the Hirsch-Fye
decoupling uses (U n_up n_dn = U (n_up n_dn - (n_up + n_dn)/2) + (U/2)(n_up + n_dn), the last
term being inside g~0), H = sum_sigma c^+_sigma h c_sigma + U (n_0up n_0dn - (n_0up + n_0dn)/2).
Everything below is the textbook many-body definition written out: Fock space of the K orbitals
x 2 spins (4^K states), fermion operators by the Jordan-Wigner sign rule, full diagonalisation,
thermal averages and the Lehmann sum of g(tau) = <T c_0(tau) c_0^+(0)> (positive convention,
g(0+) = 1 - n).
"""
from __future__ import annotations

import numpy as np


def single_particle_h(e, w):
    """K x K symmetric h with <0| (z - h)^{-1} |0> = sum_k w_k / (z - e_k): h = Q^T diag(e) Q with
    Q orthogonal and Q[k][0]^2 = w_k (first column of a QR factor of a matrix whose first column
    is sqrt(w), a unit vector)."""
    e = np.asarray(e, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    K = len(e)
    rng = np.random.default_rng(0)
    B = rng.normal(size=(K, K))
    B[:, 0] = np.sqrt(w)
    Q, _ = np.linalg.qr(B)
    return Q.T @ np.diag(e) @ Q


def _annihilators(n_modes):
    """Dense annihilation operators a_p on the 2^n_modes Fock space (Jordan-Wigner order)."""
    dim = 1 << n_modes
    ops = []
    for p in range(n_modes):
        a = np.zeros((dim, dim))
        for s in range(dim):
            if (s >> p) & 1:
                sign = -1.0 if bin(s & ((1 << p) - 1)).count("1") % 2 else 1.0
                a[s ^ (1 << p), s] = sign
        ops.append(a)
    return ops


def anderson_ed(e, w, U, beta, L):
    """Exact impurity observables of the pole bath (e, w) at interaction U and inverse temperature
    beta: returns (g[L] at tau_m = m beta / L, tau_0 = 0+, n per spin, double occupancy)."""
    h = single_particle_h(e, w)
    K = h.shape[0]
    a = _annihilators(2 * K)          # mode 2 i + s: orbital i, spin s (0 up, 1 down)
    dim = 1 << (2 * K)
    H = np.zeros((dim, dim))
    for s in (0, 1):
        for i in range(K):
            for j in range(K):
                if h[i, j] != 0.0:
                    H += h[i, j] * (a[2 * i + s].T @ a[2 * j + s])
    n_up = a[0].T @ a[0]
    n_dn = a[1].T @ a[1]
    H += U * (n_up @ n_dn - 0.5 * (n_up + n_dn))
    E, P = np.linalg.eigh(H)
    E0 = E.min()
    wgt = np.exp(-beta * (E - E0))
    Z = wgt.sum()

    def thermal(op):
        return float(np.einsum("m,m->", wgt, np.einsum("im,ij,jm->m", P, op, P)) / Z)

    n = thermal(n_up)
    d = thermal(n_up @ n_dn)
    # g(tau) = (1/Z) sum_{m,n} e^{-(beta - tau) E_m} e^{-tau E_n} |<n| c^+ |m>|^2
    cdag = P.T @ a[0].T @ P            # <n| c^+ |m> in the eigenbasis: [n, m]
    M2 = cdag ** 2
    g = np.zeros(L)
    for k in range(L):
        tau = k * beta / L
        em = np.exp(-(beta - tau) * (E - E0))
        en = np.exp(-tau * (E - E0))
        g[k] = float(en @ M2 @ em) / Z
    return g, n, d
