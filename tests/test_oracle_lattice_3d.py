"""Pins of the oracle's three-dimensional geometries (the trapped box with periodic boundaries and
the slab periodic across its layers, "Efficient simulations for three dimensions").

Each pin is fixed by something other than the oracle: closed-form tight-binding spectra, the trap
formula at given coordinates, orbit counts of the point groups counted by hand, and the exact
lattice Green function of a staggered-field Hamiltonian, whose diagonal must be constant on every
orbit (with the spin exchange of the sublattice flip) and distinct between orbits.
"""
import itertools
from math import comb

import numpy as np
import pytest

from oracle.lattice import Lattice, lattice_entries, lattice_step


def _ring(n):        # periodic chain of n sites
    return [-2.0 * np.cos(2.0 * np.pi * m / n) for m in range(n)]


def _chain(n):       # open chain of n sites
    return [-2.0 * np.cos(np.pi * m / (n + 1)) for m in range(1, n + 1)]


@pytest.mark.parametrize("L", [4, 6])
def test_free_periodic_box_spectrum(L):
    """V0 = 0, periodic box: H0 = -t A has eigenvalues -2t (cos kx + cos ky + cos kz),
    k = 2 pi m / L."""
    lat = Lattice(L, L, geometry=2, periodic=True, t=1.0, V0=0.0, Lz=L)
    ev = np.sort(np.linalg.eigvalsh(lat.H0))
    want = np.sort([a + b + c for a, b, c in itertools.product(_ring(L), _ring(L), _ring(L))])
    assert np.abs(ev - want).max() < 1e-12
    assert np.all(lat.z == 6)


def test_free_open_box_spectrum():
    lat = Lattice(3, 4, geometry=2, periodic=False, t=1.0, V0=0.0, Lz=5)
    ev = np.sort(np.linalg.eigvalsh(lat.H0))
    want = np.sort([a + b + c for a, b, c in itertools.product(_chain(3), _chain(4), _chain(5))])
    assert np.abs(ev - want).max() < 1e-12
    assert lat.z.min() == 3 and lat.z.max() == 6


@pytest.mark.parametrize("periodic", [False, True])
def test_free_slab_spectrum(periodic):
    """Slab: open (or periodic) in the plane, always periodic across the Lz = 4 layers."""
    Lx, Ly, Lz = 6, 4, 4
    lat = Lattice(Lx, Ly, geometry=3, periodic=periodic, t=1.0, V0=0.0, Lz=Lz)
    inplane = _ring if periodic else _chain
    ev = np.sort(np.linalg.eigvalsh(lat.H0))
    want = np.sort([a + b + c for a, b, c in itertools.product(inplane(Lx), inplane(Ly), _ring(Lz))])
    assert np.abs(ev - want).max() < 1e-12


def test_trap_values_and_numbering():
    box = Lattice(4, 4, geometry=2, periodic=False, V0=0.2, Lz=4)
    i = (3 * 4 + 2) * 4 + 1                       # (x, y, z) = (1, 2, 3)
    assert (box.x[i], box.y[i], box.zc[i]) == (1, 2, 3)
    assert abs(box.V[i] - 0.2 * (0.25 + 0.25 + 2.25)) < 1e-15
    assert abs(box.V[0] - 0.2 * 3 * 2.25) < 1e-15
    slab = Lattice(5, 5, geometry=3, V0=0.3, Lz=4)
    for z in range(4):                            # cylindrical: equal on every layer
        j = (z * 5 + 4) * 5 + 0                   # (0, 4, z): dx = -2, dy = 2
        assert abs(slab.V[j] - 0.3 * 8.0) < 1e-15
    assert slab.V[(2 * 5 + 2) * 5 + 2] == 0.0


@pytest.mark.parametrize("L,periodic", [(4, False), (6, False), (5, False), (4, True), (6, True)])
def test_box_orbit_counts(L, periodic):
    """Cube about its centre: an orbit of the 48 signed permutations is a multiset of three
    |d| values out of m = ceil(L/2), so there are C(m + 2, 3) of them."""
    lat = Lattice(L, L, geometry=2, periodic=periodic, V0=0.1, Lz=L)
    reps, _, _ = lat.orbits()
    m = (L + 1) // 2
    assert len(reps) == comb(m + 2, 3)
    assert len(lat._images) == 48


def test_tetragonal_box_and_slab_orbit_counts():
    box = Lattice(4, 4, geometry=2, V0=0.1, Lz=6)            # D4h: 3 planar x 3 |dz| values
    assert len(box.orbits()[0]) == 3 * 3 and len(box._images) == 16
    slab = Lattice(6, 6, geometry=3, V0=0.1, Lz=4)           # every layer equivalent
    assert len(slab.orbits()[0]) == 3 * 4 // 2 and len(slab._images) == 8 * 2 * 4
    slab2 = Lattice(6, 4, geometry=3, periodic=True, V0=0.1, Lz=4)   # no axis exchange
    assert len(slab2.orbits()[0]) == 3 * 2 and len(slab2._images) == 4 * 2 * 4


@pytest.mark.parametrize("geom,L,Lz,periodic", [(2, 4, 4, True), (2, 4, 4, False), (2, 5, 5, False),
                                                (3, 6, 4, False), (3, 4, 4, True), (2, 4, 6, False)])
def test_orbits_are_the_symmetry_classes_of_an_af_state(geom, L, Lz, periodic):
    """Exact lattice Green function of H0 plus a staggered field -sigma h eps_i: its diagonal is
    G_{i,sigma} = G_{rep(i), sigma xor flip(i)} on every site, and the unordered pair
    {G_i_up, G_i_dn} differs between orbits (no accidental degeneracy at these parameters)."""
    lat = Lattice(L, L, geometry=geom, periodic=periodic, t=1.0, V0=0.137, Lz=Lz)
    reps, rep_of, flip = lat.orbits()
    mu, beta, h = 0.9, 3.0, 0.23
    g = []
    for sg in (1.0, -1.0):
        sig = np.tile(-sg * h * lat.parity.astype(float), (3, 1)).astype(np.complex128)
        g.append(lattice_step(lat.H0, mu, beta, sig))         # [3 frequencies, N]
    g = np.array(g)                                           # [spin, freq, N]
    for i in range(lat.N):
        r = reps[rep_of[i]]
        for sp in range(2):
            assert np.abs(g[sp, :, i] - g[sp ^ flip[i], :, r]).max() < 1e-12
    pairs = {tuple(np.round(sorted([g[0, 0, r].real, g[1, 0, r].real]), 9)) for r in reps}
    assert len(pairs) == len(reps)


def test_lattice_entries_on_a_periodic_box():
    lat = Lattice(4, 4, geometry=2, periodic=True, V0=0.05, Lz=4)
    rng = np.random.default_rng(3)
    sig = rng.normal(size=lat.N) - 1j * rng.uniform(0.1, 0.5, lat.N)
    sites = [0, 21, 63]
    got = lattice_entries(lat.H0, 0.4, 5.0, sig, 7, sites)
    want = lattice_step(lat.H0, 0.4, 5.0, sig[None, :], n_index=[7])[0, sites]
    assert np.abs(got - want).max() < 1e-13
