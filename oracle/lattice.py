"""Lattice side of the oracle: geometry, trap, point-group orbits and the RDMFT lattice step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

* eq. 1 ("Model and Methods"): H = -t sum_<ij> c^+_i c_j + U sum n_up n_dn + sum (V_i - mu) n,
  V_i = V0 r_i^2 (r in lattice units a = 1).  The one-body matrix H0 = -t A + diag(V).
* eq. 2: [G(i w_n)^{-1}]_ij = t_ij + [i w_n + mu - V_i - Sigma_i(i w_n)] delta_ij with t_ij = t
  on nearest neighbours, i.e. G(i w_n) = [(i w_n + mu) 1 - H0 - diag(Sigma(i w_n))]^{-1}; only the
  site-diagonal part is kept.  Here it is literally that inverse (numpy.linalg.inv), frequency
  by frequency.
"""
from __future__ import annotations

import numpy as np


class Lattice:
    """Sites, trap potential, hopping and sublattice parity of one geometry.

    geometry 0: Lx x Ly square, site (x, y) has index y * Lx + x, centre ((Lx-1)/2, (Ly-1)/2).
    geometry 1: site-centred disc x^2 + y^2 <= R^2 (R = Lx), sites ordered by (y, x).
    geometry 2: Lx x Ly x Lz box, site (x, y, z) has index (z * Ly + y) * Lx + x, spherical trap
                V0 (dx^2 + dy^2 + dz^2) about the box centre; periodic wraps all three axes.
    geometry 3: slab of Lz layers, same numbering, cylindrical trap V0 (dx^2 + dy^2); always
                periodic across the layers, periodic also wraps x and y.
    The two three-dimensional cases follow "Efficient simulations for three dimensions": periodic
    boundaries for the trapped box, and a slab periodic perpendicular to its layers with the
    perpendicular part of the trap left out.
    """

    def __init__(self, Lx, Ly=None, geometry=0, periodic=False, t=1.0, V0=0.0, Lz=1):
        self.geometry = geometry
        self.t = float(t)
        self.V0 = float(V0)
        Ly = Lx if Ly is None else Ly
        three_d = geometry in (2, 3)
        Lz = Lz if three_d else 1
        self.Lx, self.Ly, self.Lz = Lx, Ly, Lz
        xs, ys, zs = [], [], []
        if geometry in (0, 2, 3):
            for z in range(Lz):
                for y in range(Ly):
                    for x in range(Lx):
                        xs.append(x)
                        ys.append(y)
                        zs.append(z)
            self.cx, self.cy, self.cz = (Lx - 1) / 2.0, (Ly - 1) / 2.0, (Lz - 1) / 2.0
        elif geometry == 1:
            R = Lx
            for y in range(-R, R + 1):
                for x in range(-R, R + 1):
                    if x * x + y * y <= R * R:
                        xs.append(x)
                        ys.append(y)
                        zs.append(0)
            self.cx, self.cy, self.cz = 0.0, 0.0, 0.0
        else:
            raise ValueError("geometry")
        self.x, self.y, self.zc = np.array(xs), np.array(ys), np.array(zs)
        self.dx = self.x - self.cx
        self.dy = self.y - self.cy
        self.dz = (self.zc - self.cz) if three_d else np.zeros(len(xs))
        self.N = len(self.x)
        self.r2 = self.dx ** 2 + self.dy ** 2 + (self.dz ** 2 if geometry == 2 else 0.0)
        self.V = self.V0 * self.r2
        self.parity = np.where((self.x + self.y + self.zc) % 2 == 0, 1, -1)
        index = {(int(a), int(b), int(c)): i for i, (a, b, c) in enumerate(zip(self.x, self.y, self.zc))}
        wrap_xy = periodic and geometry in (0, 2, 3)
        wrap_z = geometry == 3 or (geometry == 2 and periodic)
        steps = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)]
        if three_d:
            steps += [(0, 0, 1), (0, 0, -1)]
        A = np.zeros((self.N, self.N))
        for i in range(self.N):
            for (ddx, ddy, ddz) in steps:
                xn, yn, zn = int(self.x[i]) + ddx, int(self.y[i]) + ddy, int(self.zc[i]) + ddz
                if wrap_xy:
                    xn %= Lx
                    yn %= Ly
                if wrap_z:
                    zn %= Lz
                j = index.get((xn, yn, zn))
                if j is not None and j != i:
                    A[i, j] = 1.0
        self.adjacency = A
        self.z = A.sum(axis=1)  # number of neighbours of each site
        self.H0 = -self.t * A + np.diag(self.V)
        self._index = index

    # --- point-group orbits ------------------------------------------------
    def _operations(self):
        """Candidate maps of the integer coordinates: signed axis permutations about the trap
        centre (the 8 planar ones in two dimensions, all 48 for the box), and for the slab the 8
        planar ones combined with z -> +-z + c (mod Lz).  Each returns (x, y, z) or None when
        the image is not a lattice point."""
        planar = [(0, 1, 2), (1, 0, 2)]
        if self.geometry == 2:
            perms = [(0, 1, 2), (1, 0, 2), (0, 2, 1), (2, 1, 0), (1, 2, 0), (2, 0, 1)]
        else:
            perms = planar
        zsigns = (1, -1) if self.geometry in (2, 3) else (1,)
        shifts = range(self.Lz) if self.geometry == 3 else (0,)
        centre = (self.cx, self.cy, self.cz)
        ops = []
        for perm in perms:
            for sx in (1, -1):
                for sy in (1, -1):
                    for sz in zsigns:
                        for c in shifts:
                            ops.append((perm, (sx, sy, sz), c))

        def apply(op, i):
            perm, sg, c = op
            d = (self.dx[i], self.dy[i], self.dz[i])
            out = []
            for a in range(2):
                v = sg[a] * d[perm[a]] + centre[a]
                if abs(v - round(v)) > 1e-9:
                    return None
                out.append(int(round(v)))
            if self.geometry == 3:
                out.append((sg[2] * int(self.zc[i]) + c) % self.Lz)
            else:
                v = sg[2] * d[perm[2]] + centre[2]
                if abs(v - round(v)) > 1e-9:
                    return None
                out.append(int(round(v)))
            return tuple(out)

        return ops, apply

    def orbits(self):
        """Inequivalent sites under the point group of the trap and the lattice.

        The operations of _operations() are kept if they map the site set onto itself.  Returns
        (reps, rep_of, flip): reps = sorted site indices of the orbit representatives; rep_of[i]
        = position in reps of the orbit of site i; flip[i] = 1 if site i and its representative
        lie on different sublattices.  An antiferromagnetic state then satisfies
        G_{i,sigma} = G_{rep, sigma xor flip}.
        """
        ops, apply = self._operations()
        images = []
        for op in ops:
            img = []
            for i in range(self.N):
                c = apply(op, i)
                j = None if c is None else self._index.get(c)
                if j is None:
                    break
                img.append(j)
            if len(img) == self.N:
                images.append(np.array(img))
        rep_site = np.array([min(int(im[i]) for im in images) for i in range(self.N)])
        reps = np.array(sorted(set(rep_site.tolist())))
        pos = {int(r): k for k, r in enumerate(reps)}
        rep_of = np.array([pos[int(r)] for r in rep_site])
        flip = (self.parity != self.parity[rep_site]).astype(np.int64)
        self._images = images
        return reps, rep_of, flip


def matsubara(beta, nw):
    """Fermionic Matsubara frequencies w_n = (2n + 1) pi T, n = 0..nw-1."""
    return (2.0 * np.arange(nw) + 1.0) * np.pi / beta


def lattice_step(H0, mu, beta, sigma, n_index=None):
    """eq. 2: site-diagonal G_ii(i w_n) of [(i w_n + mu) 1 - H0 - diag(Sigma(i w_n))]^{-1}.

    sigma: [k, N] complex (one spin), the self-energy at the frequencies n_index (default
    n = 0..k-1).  Returns [k, N] complex.
    """
    k, N = sigma.shape
    n_index = np.arange(k) if n_index is None else np.asarray(n_index)
    w = (2.0 * n_index + 1.0) * np.pi / beta
    out = np.zeros((k, N), dtype=np.complex128)
    eye = np.eye(N)
    for q in range(k):
        M = (1j * w[q] + mu) * eye - H0 - np.diag(sigma[q])
        out[q] = np.diag(np.linalg.inv(M))
    return out


def lattice_entries(H0, mu, beta, sigma_row, n, sites):
    """eq. 2 at one frequency for large lattices: G_ii(i w_n) for the listed sites i only, each as
    entry i of the column x = M^{-1} e_i of M = (i w_n + mu) 1 - H0 - diag(Sigma(i w_n)), from one
    sparse LU factorisation of M (a library solve; M has at most five nonzeros per row).

    sigma_row: [N] complex, the self-energy of every site at w_n.  Returns [len(sites)] complex.
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    N = H0.shape[0]
    w = (2.0 * n + 1.0) * np.pi / beta
    M = sp.csc_matrix(((1j * w + mu) * sp.identity(N, dtype=np.complex128)
                       - sp.csc_matrix(H0) - sp.diags(np.asarray(sigma_row))).astype(np.complex128))
    lu = spla.splu(M)
    out = np.zeros(len(sites), dtype=np.complex128)
    for k, i in enumerate(sites):
        e = np.zeros(N, dtype=np.complex128)
        e[i] = 1.0
        out[k] = lu.solve(e)[i]
    return out
