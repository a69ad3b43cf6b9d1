"""Pins of the exact-diagonalisation oracle, and the Hirsch-Fye discretisation against it: the
exact brute-force Hirsch-Fye averages at finite dtau, extrapolated to dtau -> 0 (errors even in
dtau), reproduce the exact continuous-time impurity."""
import numpy as np
import pytest

import oracle as o
from oracle.ed import anderson_ed, single_particle_h
from paper_1006_2716_gb300 import workloads as wl


def test_single_particle_h_has_the_pole_spectrum():
    e, w = wl.bath_poles(3)
    h = single_particle_h(e, w)
    assert np.allclose(h, h.T)
    for z in (0.3 + 1.1j, -2.0 + 0.2j):
        assert abs(np.linalg.inv(z * np.eye(len(e)) - h)[0, 0] - (w / (z - e)).sum()) < 1e-14


def test_u0_is_the_free_bath():
    e, w = wl.bath_poles(7)
    beta, L = 3.0, 16
    g, n, d = anderson_ed(e, w, 0.0, beta, L)
    assert np.abs(g - wl.pole_bath_tau(beta, L, e, w)).max() < 1e-12
    f = 1.0 / (np.exp(beta * e) + 1.0)
    assert abs(n - (w * f).sum()) < 1e-12
    assert abs(d - n * n) < 1e-12          # U = 0: the two spins are independent


@pytest.mark.parametrize("eps,U,beta", [(-1.3, 4.0, 4.0), (0.4, 2.0, 5.0)])
def test_single_level_is_the_atom(eps, U, beta):
    # one pole at the Hartree-shifted level eps + U/2 is the atom with level eps
    L = 12
    g, n, d = anderson_ed([eps + U / 2.0], [1.0], U, beta, L)
    tau = np.arange(L) * beta / L
    Z = 1 + 2 * np.exp(-beta * eps) + np.exp(-beta * (2 * eps + U))
    assert abs(n - (np.exp(-beta * eps) + np.exp(-beta * (2 * eps + U))) / Z) < 1e-12
    assert abs(d - np.exp(-beta * (2 * eps + U)) / Z) < 1e-12
    want = (np.exp(-eps * tau) + np.exp(-beta * eps) * np.exp(-(eps + U) * tau)) / Z
    assert np.abs(g - want).max() < 1e-12


def test_particle_hole_symmetric_bath():
    e = np.array([-1.7, -0.4, 0.4, 1.7])
    w = np.array([0.2, 0.3, 0.3, 0.2])
    beta, L, U = 4.0, 16, 3.0
    g, n, d = anderson_ed(e, w, U, beta, L)
    assert abs(n - 0.5) < 1e-12
    tau = np.arange(1, L)
    g_full = np.append(g, 1.0 - g[0])         # g(beta^-) = 1 - g(0+) = n
    assert np.abs(g_full[tau] - g_full[L - tau]).max() < 1e-12


@pytest.mark.parametrize("seed,beta,U", [(3, 2.0, 2.0), (5, 2.0, 3.0)])
def test_hirsch_fye_extrapolates_to_exact(seed, beta, U):
    """Brute force over all 2^L fields (exact at each dtau = beta / L, L = 8..16), fitted as
    a + b dtau^2 + c dtau^4: a is the exact double occupancy of the continuous-time impurity."""
    e, w = wl.bath_poles(seed)
    _, n_ed, d_ed = anderson_ed(e, w, U, beta, 8)
    Ls = [8, 10, 12, 14, 16]
    d = []
    for L in Ls:
        g0 = o.build_g0(wl.pole_bath_tau(beta, L, e, w))
        _, lam = o.constants(beta, U, L)
        d.append(o.brute_force(lam, g0, g0)[2 * L + 2])
    dt = beta / np.array(Ls, dtype=float)
    A = np.stack([np.ones_like(dt), dt ** 2, dt ** 4], axis=1)
    coef, *_ = np.linalg.lstsq(A, np.array(d), rcond=None)
    assert abs(d[-1] - d_ed) > 3e-4             # the discretisation error is visible ...
    assert abs(coef[0] - d_ed) < 1e-5           # ... and extrapolates away
