"""Pins of the oracle's lattice step (eq. 2), C4v reduction and tau <-> i w transforms.

CPU only.  References independent of the oracle: numpy eigendecomposition (a different library
routine than the inverse the oracle uses), closed-form free-fermion Green functions, exact
Fourier integrals of polynomials, symmetry of the Hamiltonian.
"""
import numpy as np
import pytest

from oracle import fourier as F
from oracle.lattice import Lattice, lattice_entries, lattice_step, matsubara


@pytest.mark.parametrize("Lx,geom,expect", [(6, 0, 6), (20, 0, 55), (30, 0, 120), (8, 1, None)])
def test_orbit_counts_and_symmetry(Lx, geom, expect):
    lat = Lattice(Lx, geometry=geom, V0=0.07)
    reps, rep_of, flip = lat.orbits()
    if expect is not None:
        assert len(reps) == expect
    # every orbit member has the trap potential and the neighbour count of its representative
    assert np.allclose(lat.V, lat.V[reps][rep_of])
    assert np.array_equal(lat.z, lat.z[reps][rep_of])
    # a sublattice flip happens exactly when parities differ
    assert np.array_equal(flip, (lat.parity != lat.parity[reps][rep_of]).astype(int))
    if geom == 0 and Lx % 2 == 0:
        assert flip.sum() == lat.N // 2       # even L: bond-centred, half the sites flip
    if geom == 1:
        assert flip.sum() == 0                # site-centred disc keeps the sublattice


def test_disc_counts():
    lat = Lattice(40, geometry=1)
    reps, _, _ = lat.orbits()
    assert lat.N == 5025 and len(reps) == 663


def test_h0_hopping_and_trap():
    lat = Lattice(6, V0=0.1)
    # corner sites have 2 neighbours, edges 3, bulk 4; V = V0 r^2 from (2.5, 2.5)
    assert lat.z[0] == 2 and lat.z[1] == 3 and lat.z[7] == 4
    assert abs(lat.V[0] - 0.1 * (2.5 ** 2 * 2)) < 1e-15
    assert np.allclose(lat.H0, lat.H0.T)
    assert np.all(np.linalg.eigvalsh(-lat.adjacency) >= -4 - 1e-12)


@pytest.mark.parametrize("Lx", [4, 6])
def test_lattice_step_free_vs_eigh(Lx):
    # U = 0, Sigma = 0: G_ii(i w) = sum_k |psi_k(i)|^2 / (i w + mu - e_k)
    lat = Lattice(Lx, V0=0.1)
    beta, mu, nw = 4.0, 0.7, 40
    G = lattice_step(lat.H0, mu, beta, np.zeros((nw, lat.N), dtype=complex))
    e, v = np.linalg.eigh(lat.H0)
    w = matsubara(beta, nw)
    ref = np.array([(np.abs(v) ** 2 / (1j * wn + mu - e)[None, :]).sum(axis=1) for wn in w])
    assert np.abs(G - ref).max() < 1e-12


def test_lattice_step_static_sigma_vs_eigh():
    # a static site-dependent real Sigma is part of the one-body matrix
    lat = Lattice(6, V0=0.1)
    beta, mu, nw = 4.0, 2.0, 20
    rng = np.random.default_rng(1)
    sig = rng.uniform(1.5, 2.5, lat.N)
    G = lattice_step(lat.H0, mu, beta, np.tile(sig.astype(complex), (nw, 1)))
    e, v = np.linalg.eigh(lat.H0 + np.diag(sig))
    w = matsubara(beta, nw)
    ref = np.array([(np.abs(v) ** 2 / (1j * wn + mu - e)[None, :]).sum(axis=1) for wn in w])
    assert np.abs(G - ref).max() < 1e-12


def _free_tau(beta, L, e, wts):
    tau = np.arange(L + 1) * beta / L
    out = np.zeros(L + 1)
    for ek, wk in zip(e, wts):
        out += wk * np.exp(-ek * tau) / (1 + np.exp(-beta * ek))
    return out


def _trunc_bound(beta, nw, c4):
    # |G - tail| <= c4 / w^4 (1 + small) beyond the cutoff; 2T sum_{n>=nw} 1/w_n^4 bound
    n = np.arange(nw, nw + 200000)
    wn = (2 * n + 1) * np.pi / beta
    return 2.0 / beta * np.sum(2.0 * c4 / wn ** 4)


@pytest.mark.parametrize("beta,eps", [(4.0, 0.8), (8.0, -1.5), (16.0, 0.0)])
def test_iw_to_tau_single_pole(beta, eps):
    nw, L = 500, 32
    G = 1.0 / (1j * matsubara(beta, nw) - eps)
    g = F.iw_to_tau(beta, G, eps, eps ** 2, L)
    ref = _free_tau(beta, L, [eps], [1.0])
    assert np.abs(g - ref).max() < _trunc_bound(beta, nw, abs(eps) ** 3 + 1e-3)


def test_iw_to_tau_two_pole_tail_coefficients():
    # G = 1/(i w - ed - V^2/(i w - eb)): c2 = ed, c3 = ed^2 + V^2 (the Weiss-field tail)
    beta, nw, L = 8.0, 500, 40
    ed, eb, V = 0.9, -0.6, 0.8
    h = np.array([[ed, V], [V, eb]])
    e, v = np.linalg.eigh(h)
    wts = np.abs(v[0]) ** 2
    iw = 1j * matsubara(beta, nw)
    G = 1.0 / (iw - ed - V ** 2 / (iw - eb))
    g = F.iw_to_tau(beta, G, ed, ed ** 2 + V ** 2, L)
    ref = _free_tau(beta, L, e, wts)
    c4 = np.sum(wts * np.abs(e) ** 3)
    assert np.abs(g - ref).max() < _trunc_bound(beta, nw, c4)
    # dropping c3 leaves an O(1/w_N^2) error outside that bound; a flipped c2 is far outside
    bad = F.iw_to_tau(beta, G, ed, 0.0, L)
    assert np.abs(bad - ref).max() > 3 * _trunc_bound(beta, nw, c4)
    bad = F.iw_to_tau(beta, G, -ed, ed ** 2 + V ** 2, L)
    assert np.abs(bad - ref).max() > 1e3 * _trunc_bound(beta, nw, c4)


def test_spline_fourier_exact_for_linear():
    # natural spline reproduces a(1 - 2 tau/beta) exactly; its transform is 4a/(beta (i w)^2)
    beta, L, nw, a = 5.0, 20, 300, 0.37
    tau = np.arange(L + 1) * beta / L
    dg = a * (1 - 2 * tau / beta)
    got = F.spline_fourier(beta, dg, nw)
    iw = 1j * matsubara(beta, nw)
    assert np.abs(got - 4 * a / (beta * iw ** 2)).max() < 1e-12


def test_natural_spline_interpolates_and_is_c2():
    rng = np.random.default_rng(3)
    y = rng.normal(size=17)
    h = 0.3
    a, b, c, d = F.natural_spline_coeffs(h, y)
    # values at both knots, continuity of first and second derivative, natural ends
    assert np.allclose(a, y[:-1], atol=1e-14)
    assert np.allclose(a + b * h + c * h ** 2 + d * h ** 3, y[1:], atol=1e-13)
    assert np.allclose(b[1:], b[:-1] + 2 * c[:-1] * h + 3 * d[:-1] * h ** 2, atol=1e-12)
    assert np.allclose(2 * c[1:], 2 * c[:-1] + 6 * d[:-1] * h, atol=1e-12)
    assert abs(c[0]) < 1e-15 and abs(2 * c[-1] + 6 * d[-1] * h) < 1e-12


def test_tau_to_iw_converges_to_exact():
    # g_ref = free level, g = another free level: G(i w) error falls with the grid spacing
    beta, nw = 6.0, 200
    iw = 1j * matsubara(beta, nw)
    e0, e1 = 0.4, 0.1
    errs = []
    for L in (16, 32, 64):
        g_ref = _free_tau(beta, L, [e0], [1.0])[:L]
        g = _free_tau(beta, L, [e1], [1.0])[:L]
        got = F.tau_to_iw(beta, g, g_ref, 1.0 / (iw - e0))
        errs.append(np.abs(got - 1.0 / (iw - e1)).max())
    assert errs[1] < 0.3 * errs[0] and errs[2] < 0.3 * errs[1]
    assert errs[2] < 2e-4


def test_tau_to_iw_identity_when_equal():
    beta, L, nw = 4.0, 16, 100
    g = _free_tau(beta, L, [0.3], [1.0])[:L]
    ref = 1.0 / (1j * matsubara(beta, nw) - 0.3)
    assert np.abs(F.tau_to_iw(beta, g, g, ref) - ref).max() == 0.0


def test_density_from_lattice_step_and_tail():
    # pin of lattice step + transform together: n_i = g_ii(beta-) of the free trapped lattice
    lat = Lattice(6, V0=0.1)
    beta, mu, nw, L = 4.0, 1.0, 500, 16
    G = lattice_step(lat.H0, mu, beta, np.zeros((nw, lat.N), dtype=complex))
    e, v = np.linalg.eigh(lat.H0)
    f = 1.0 / (1.0 + np.exp(beta * (e - mu)))
    nref = (np.abs(v) ** 2 * f[None, :]).sum(axis=1)
    for i in (0, 7, 14):
        c2 = lat.V[i] - mu
        c3 = c2 ** 2 + lat.z[i]
        g = F.iw_to_tau(beta, G[:, i], c2, c3, L)
        c4 = np.abs(np.linalg.matrix_power(lat.H0 - mu * np.eye(lat.N), 3)[i, i]) + 10
        assert abs(g[L] - nref[i]) < _trunc_bound(beta, nw, c4)
        assert abs(g[0] - (1 - nref[i])) < _trunc_bound(beta, nw, c4)


@pytest.mark.parametrize("Lx,geom", [(6, 0), (6, 1)])
def test_lattice_entries_match_the_inverse_and_eigh(Lx, geom):
    """One column of M^{-1} per sampled site (sparse LU) equals the diagonal of the dense inverse
    for an arbitrary causal self-energy, and the eigenvector sum for a static one."""
    lat = Lattice(Lx, geometry=geom, V0=0.08)
    beta, mu, N = 5.0, 1.3, lat.N
    rng = np.random.default_rng(11 + geom)
    sites = sorted(rng.choice(N, 5, replace=False))
    for n in (0, 3, 40):
        sig = 0.4 + rng.uniform(-0.5, 0.5, N) - 1j * rng.uniform(0.05, 0.6, N)
        dense = lattice_step(lat.H0, mu, beta, sig[None, :], n_index=[n])[0]
        got = lattice_entries(lat.H0, mu, beta, sig, n, sites)
        assert np.abs(got - dense[sites]).max() < 1e-12 * np.abs(dense).max()
    # static self-energy s: G_ii = sum_k |psi_k(i)|^2 / (i w_n + mu - s - e_k)
    s0 = 0.7
    e, psi = np.linalg.eigh(lat.H0)
    for n in (0, 9):
        w = (2 * n + 1) * np.pi / beta
        want = (np.abs(psi[sites]) ** 2 / (1j * w + mu - s0 - e)[None, :]).sum(axis=1)
        got = lattice_entries(lat.H0, mu, beta, np.full(N, s0, dtype=complex), n, sites)
        assert np.abs(got - want).max() < 1e-12
