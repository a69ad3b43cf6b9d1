"""Pins of the oracle's Hirsch-Fye core against what the method and the mathematics fix.

Each test pins the oracle to something other than itself: published known-answer vectors,
closed forms (free atom, atomic limit), determinants computed by a different algorithm, exact
enumeration, symmetries.  CPU only.
"""
import os

import numpy as np
import pytest

import oracle as o
from paper_1006_2716_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert list(o.philox4x32_10(ctr, key)) == expect


def test_uniform_mapping_and_keying():
    # u = ((x0 << 32 | x1) >> 11) 2^-53 with counter (sweep, l, chain, site), key (lo, hi)
    seed = 0x0123456789ABCDEF
    x = o.philox4x32_10([7, 3, 5, 11], [seed & 0xFFFFFFFF, seed >> 32])
    bits = ((int(x[0]) << 32) | int(x[1])) >> 11
    assert o.uniform(seed, 11, 5, 7, 3) == bits / 2.0 ** 53
    us = np.array([o.uniform(9, 0, 0, sw, l) for sw in range(50) for l in range(40)])
    assert us.min() >= 0.0 and us.max() < 1.0
    assert abs(us.mean() - 0.5) < 0.03


def test_init_fields_top_bit():
    s = o.init_fields(5, 2, 3, 64)
    for l in range(64):
        x = o.philox4x32_10([0xFFFFFFFF, l, 3, 2], [5, 0])
        assert s[l] == (-1 if x[0] >> 31 else 1)
    assert set(np.unique(s)) <= {-1, 1}


def test_constants_closed_form():
    # cosh(lambda) = exp(dtau U / 2); at dtau = 0.25: lambda = acosh(e^0.5) = 1.08504 (U = 4)
    # and acosh(e^1) = 1.65745 (U = 8)
    dt, lam = o.constants(4.0, 4.0, 16)
    assert dt == 0.25
    assert abs(np.cosh(lam) - np.exp(0.5)) < 1e-14
    assert abs(lam - 1.08504) < 5e-6
    _, lam8 = o.constants(8.0, 8.0, 32)
    assert abs(lam8 - 1.65745) < 5e-6


@pytest.mark.parametrize("L,beta,et", [(8, 4.0, 0.7), (16, 4.0, -1.1), (32, 8.0, 0.0)])
def test_g0_is_inverse_of_free_atom_bss_matrix(L, beta, et):
    # For one free level the discretised propagator is the inverse of the antiperiodic
    # bidiagonal matrix O: O_ll = 1, O_{l,l-1} = -B, O_{0,L-1} = +B, B = exp(-dtau et).
    dt = beta / L
    g0 = o.build_g0(wl.pole_bath_tau(beta, L, [et], [1.0]))
    B = np.exp(-dt * et)
    O = np.eye(L)
    for l in range(1, L):
        O[l, l - 1] = -B
    O[0, L - 1] = B
    assert np.abs(g0 @ O - np.eye(L)).max() < 1e-13


def test_u0_gives_g0_bitwise():
    L, beta = 16, 4.0
    gt = wl.random_baths(3, 1, beta, L)[0]
    g0u, g0d = o.build_g0(gt[0]), o.build_g0(gt[1])
    _, lam = o.constants(beta, 0.0, L)
    assert lam == 0.0
    s = o.init_fields(1, 0, 0, L)
    Gu, _ = o.dyson(g0u, s, 1, lam)
    Gd, _ = o.dyson(g0d, s, -1, lam)
    assert np.array_equal(Gu, g0u) and np.array_equal(Gd, g0d)
    s0 = s.copy()
    for sw in range(5):
        acc = o.sweep(lam, 1, 0, 0, sw, s, Gu, Gd)
        assert acc == L                          # R = 1 > u always
    assert np.array_equal(s, s0 * (-1) ** 5)
    assert np.array_equal(Gu, g0u) and np.array_equal(Gd, g0d)


@pytest.mark.parametrize("L", [8, 16, 32])
def test_ratio_equals_determinant_ratio(L):
    beta, U = 0.25 * L, 6.0
    gt = wl.random_baths(11, 1, beta, L)[0]
    g0 = [o.build_g0(gt[0]), o.build_g0(gt[1])]
    _, lam = o.constants(beta, U, L)
    s = o.init_fields(4, 0, 0, L)
    Gu, du = o.dyson(g0[0], s, 1, lam)
    Gd, dd = o.dyson(g0[1], s, -1, lam)
    for l in range(0, L, 3):
        p, a, R = o.ratio(lam, s, l, Gu, Gd)
        s2 = s.copy()
        s2[l] = -s2[l]
        _, du2 = o.dyson(g0[0], s2, 1, lam)
        _, dd2 = o.dyson(g0[1], s2, -1, lam)
        assert abs(R[0] - du2 / du) < 1e-11 * abs(du2 / du)
        assert abs(R[1] - dd2 / dd) < 1e-11 * abs(dd2 / dd)
        assert abs(p - (du2 * dd2) / (du * dd)) < 1e-10 * abs(p)


@pytest.mark.parametrize("L", [16, 32, 64])
def test_sherman_morrison_matches_recompute(L):
    beta, U = 0.25 * L, 8.0
    gt = wl.random_baths(5, 1, beta, L)[0]
    g0u, g0d = o.build_g0(gt[0]), o.build_g0(gt[1])
    _, lam = o.constants(beta, U, L)
    s = o.init_fields(2, 0, 0, L)
    Gu, _ = o.dyson(g0u, s, 1, lam)
    Gd, _ = o.dyson(g0d, s, -1, lam)
    total = 0
    for sw in range(4):
        total += o.sweep(lam, 2, 0, 0, sw, s, Gu, Gd)
        Ru, _ = o.dyson(g0u, s, 1, lam)
        Rd, _ = o.dyson(g0d, s, -1, lam)
        assert np.abs(Gu - Ru).max() < 1e-12 * np.abs(Ru).max()
        assert np.abs(Gd - Rd).max() < 1e-12 * np.abs(Rd).max()
    assert total > 0


def _atomic(beta, U, eps, L):
    tau = np.arange(L) * beta / L
    Z = 1 + 2 * np.exp(-beta * eps) + np.exp(-beta * (2 * eps + U))
    n = (np.exp(-beta * eps) + np.exp(-beta * (2 * eps + U))) / Z
    d = np.exp(-beta * (2 * eps + U)) / Z
    g = (np.exp(-eps * tau) + np.exp(-beta * eps) * np.exp(-(eps + U) * tau)) / Z
    return g, n, d


@pytest.mark.parametrize("L,beta,U,eps", [(8, 4.0, 4.0, -1.3), (12, 3.0, 6.0, -3.0),
                                          (10, 5.0, 2.0, 0.4)])
def test_brute_force_atomic_limit_exact(L, beta, U, eps):
    # t = 0: all Trotter factors commute, Hirsch-Fye is exact; bath = free level at eps + U/2
    _, lam = o.constants(beta, U, L)
    gt = wl.pole_bath_tau(beta, L, [eps + U / 2.0], [1.0])
    g0 = o.build_g0(gt)
    out = o.brute_force(lam, g0, g0)
    g, n, d = _atomic(beta, U, eps, L)
    assert np.abs(out[:L] - g).max() < 1e-12
    assert np.abs(out[L:2 * L] - g).max() < 1e-12
    assert abs(out[2 * L] - n) < 1e-12 and abs(out[2 * L + 1] - n) < 1e-12
    assert abs(out[2 * L + 2] - d) < 1e-12


@pytest.mark.parametrize("L", [8, 12])
def test_brute_force_particle_hole_symmetry(L):
    # symmetric bath (poles +-e with equal weights) at half filling: n = 1/2 per spin and
    # g(tau) = g(beta - tau) exactly
    beta, U = 0.3 * L, 5.0
    gt = wl.pole_bath_tau(beta, L, [-1.2, 1.2, -0.4, 0.4], [0.2, 0.2, 0.3, 0.3])
    g0 = o.build_g0(gt)
    _, lam = o.constants(beta, U, L)
    out = o.brute_force(lam, g0, g0)
    for sp in range(2):
        g = out[sp * L:(sp + 1) * L]
        assert abs(out[2 * L + sp] - 0.5) < 1e-12
        assert abs(g[0] - 0.5) < 1e-12
        for m in range(1, L):
            assert abs(g[m] - g[L - m]) < 1e-12


def _qmc(L, beta, U, g0u, g0d, sweeps, chains=4, seed=7, bin_size=250):
    _, lam = o.constants(beta, U, L)
    W = 2 * L + 3
    nb = sweeps // bin_size
    xs = []
    for c in range(chains):
        s = o.init_fields(seed, 0, c, L)
        Gu, _ = o.dyson(g0u, s, 1, lam)
        Gd, _ = o.dyson(g0d, s, -1, lam)
        bins = np.zeros((nb, W))
        o.run_chain(lam, g0u, g0d, seed, 0, c, 0, 200, sweeps, 10, bin_size, s, Gu, Gd, bins)
        xs.append(bins / bin_size)
    x = np.concatenate(xs)
    return x.mean(axis=0), x.std(axis=0, ddof=1) / np.sqrt(x.shape[0])


def test_qmc_matches_brute_force_spin_asymmetric_bath():
    # a chain that swapped spins, signs or slices would sample a different distribution
    L, beta, U = 8, 2.0, 4.0
    gt = wl.random_baths(21, 1, beta, L)[0]
    g0u, g0d = o.build_g0(gt[0]), o.build_g0(gt[1])
    _, lam = o.constants(beta, U, L)
    exact = o.brute_force(lam, g0u, g0d)
    mean, err = _qmc(L, beta, U, g0u, g0d, 20000)
    z = np.abs(mean - exact) / np.maximum(err, 1e-15)
    assert np.max(z) < 4.5, (np.max(z), np.argmax(z))
    # the two spins really differ here
    assert abs(exact[2 * L] - exact[2 * L + 1]) > 0.02


def test_qmc_atomic_limit_within_error():
    L, beta, U, eps = 16, 4.0, 4.0, -1.7
    gt = wl.pole_bath_tau(beta, L, [eps + U / 2.0], [1.0])
    g0 = o.build_g0(gt)
    mean, err = _qmc(L, beta, U, g0, g0, 10000)
    g, n, d = _atomic(beta, U, eps, L)
    exact = np.concatenate([g, g, [n, n, d]])
    z = np.abs(mean - exact) / np.maximum(err, 1e-15)
    assert np.max(z) < 4.5


@pytest.mark.parametrize("stagger,refresh_at", [(0, (10, 20, 30)), (1, (7, 17, 27))])
def test_run_chain_refresh_and_bins(stagger, refresh_at):
    # cadence: a refresh exactly when the sweep counter hits a multiple of refresh_every
    # (staggered: site 1 + chain 2 moves the counter by 3, so the refreshes come after sweeps
    # 7, 17, 27); bins hold sums of bin_size measurements
    L, beta, U = 16, 4.0, 4.0
    gt = wl.random_baths(8, 1, beta, L)[0]
    g0u, g0d = o.build_g0(gt[0]), o.build_g0(gt[1])
    _, lam = o.constants(beta, U, L)
    s = o.init_fields(3, 1, 2, L)
    Gu, _ = o.dyson(g0u, s, 1, lam)
    Gd, _ = o.dyson(g0d, s, -1, lam)
    bins = np.zeros((3, 2 * L + 3))
    acc, nsw = o.run_chain(lam, g0u, g0d, 3, 1, 2, 0, 5, 30, 10, 10, s, Gu, Gd, bins,
                           refresh_stagger=stagger)
    assert nsw == 35
    # replay by hand from a copy
    s2 = o.init_fields(3, 1, 2, L)
    Hu, _ = o.dyson(g0u, s2, 1, lam)
    Hd, _ = o.dyson(g0d, s2, -1, lam)
    acc2 = 0
    ref = np.zeros((3, 2 * L + 3))
    for k in range(35):
        acc2 += o.sweep(lam, 3, 1, 2, k, s2, Hu, Hd)
        if k + 1 in refresh_at:
            Hu, _ = o.dyson(g0u, s2, 1, lam)
            Hd, _ = o.dyson(g0d, s2, -1, lam)
        if k >= 5:
            ref[(k - 5) // 10] += o.measure(Hu, Hd)
    assert acc == acc2
    assert np.array_equal(s, s2)
    assert np.abs(bins - ref).max() < 1e-13
    assert np.array_equal(Gu, Hu) and np.array_equal(Gd, Hd)
    # a measurement is an average of L diagonals: density = 1 - G(0+)
    m = o.measure(Hu, Hd)
    assert abs(m[2 * L] - (1 - m[0])) < 1e-14


def test_tie_watch_counts_without_changing_results():
    # the near-tie watch is instrumentation: with it on, every decision and every G entry are
    # those of an unwatched run; a huge window counts every proposal, a zero window none
    L, beta, U = 16, 4.0, 4.0
    b = wl.random_baths(11, 1, beta, L)[0]
    _, lam = o.constants(beta, U, L)
    g0u, g0d = o.build_g0(b[0]), o.build_g0(b[1])

    def run(rel):
        o.tie_watch(rel)
        s = o.init_fields(5, 0, 0, L)
        Gu, _ = o.dyson(g0u, s, 1, lam)
        Gd, _ = o.dyson(g0d, s, -1, lam)
        acc = sum(o.sweep(lam, 5, 0, 0, k, s, Gu, Gd) for k in range(6))
        n = o.tie_count()
        o.tie_watch(0.0)
        return acc, s, Gu, Gd, n

    a0, s0, u0, d0, n0 = run(0.0)
    a1, s1, u1, d1, n1 = run(1e300)
    assert n0 == 0 and n1 == 6 * L
    assert a0 == a1 and np.array_equal(s0, s1)
    assert np.array_equal(u0, u1) and np.array_equal(d0, d1)
    _, _, _, _, n2 = run(1e-3)
    assert 0 <= n2 <= 6 * L
