"""Pins of the oracle's free-fermion thermodynamics (the U = 0 reference for the entropy obtained
from dS/dmu = dN/dT, "Results for square lattice"), and the host-side Simpson integration of the
scan.  No GPU."""
import numpy as np
import pytest

from oracle import thermo as ot
from oracle.lattice import Lattice
from paper_1006_2716_gb300.thermo import cumulative_simpson


def test_single_level_closed_forms():
    """One site, one level e: N = 2 f, S = 2 (-f ln f - (1-f) ln(1-f)), f = 1/(e^{(e-mu)/T}+1)."""
    H0 = np.array([[0.7]])
    for mu, T in ((0.0, 0.3), (1.5, 2.0), (0.7, 0.5)):
        f = 1.0 / (np.exp((0.7 - mu) / T) + 1.0)
        assert abs(ot.free_density(H0, mu, T)[0] - 2 * f) < 1e-15
        want = 2 * (-f * np.log(f) - (1 - f) * np.log(1 - f))
        assert abs(ot.free_entropy(H0, mu, T)[0] - want) < 1e-14
    assert abs(ot.free_entropy(H0, 0.7, 1.0)[0] - 2 * np.log(2.0)) < 1e-15


@pytest.mark.parametrize("geom,L", [(0, 6), (1, 4), (2, 4)])
def test_maxwell_relation_and_derivative(geom, L):
    """dS/dmu (central difference of the closed-form S) equals the closed-form dN/dT, site by
    site, and dN/dT equals the central difference of N in T."""
    lat = Lattice(L, L, geometry=geom, V0=0.1, Lz=L)
    T, mu, h = 0.6, -0.8, 1e-4
    dsdmu = (ot.free_entropy(lat.H0, mu + h, T) - ot.free_entropy(lat.H0, mu - h, T)) / (2 * h)
    dndT = ot.free_dndT(lat.H0, mu, T)
    assert np.abs(dsdmu - dndT).max() < 1e-7
    fd = (ot.free_density(lat.H0, mu, T + h) - ot.free_density(lat.H0, mu, T - h)) / (2 * h)
    assert np.abs(fd - dndT).max() < 1e-7


def test_limits():
    lat = Lattice(6, 6, V0=0.1)
    assert ot.free_entropy(lat.H0, -40.0, 0.5).sum() < 1e-20          # empty
    assert ot.free_density(lat.H0, -40.0, 0.5).sum() < 1e-20
    # T -> infinity: every level half filled per spin, S -> 2 N ln 2, n_i -> 1
    S = ot.free_entropy(lat.H0, 0.0, 1e6)
    assert np.abs(S - 2 * np.log(2.0)).max() < 1e-9
    assert np.abs(ot.free_density(lat.H0, 0.0, 1e6) - 1.0).max() < 1e-6
    # local entropies sum to the total of the level picture
    e = np.linalg.eigvalsh(lat.H0)
    f = 1.0 / (np.exp((e - 0.3) / 0.7) + 1.0)
    total = 2 * np.sum(-f * np.log(f) - (1 - f) * np.log(1 - f))
    assert abs(ot.free_entropy(lat.H0, 0.3, 0.7).sum() - total) < 1e-12


def test_cumulative_simpson():
    """Exact for cubics; cumulative values at the even points; errors on bad grids."""
    mus = np.linspace(-2.0, 3.0, 11)
    y = 2 * mus ** 3 - mus ** 2 + 4
    F = lambda x: 0.5 * x ** 4 - x ** 3 / 3 + 4 * x
    got = cumulative_simpson(mus, y)
    assert np.abs(got - (F(mus[0::2]) - F(mus[0]))).max() < 1e-12
    two = cumulative_simpson(mus, np.stack([y, 3 * y]))
    assert two.shape == (2, 6) and np.abs(two[1] - 3 * got).max() < 1e-12
    with pytest.raises(ValueError):
        cumulative_simpson(np.linspace(0, 1, 10), np.zeros(10))
    with pytest.raises(ValueError):
        cumulative_simpson(np.array([0.0, 0.1, 0.3]), np.zeros(3))
