"""Lattice side of the oracle: geometry, trap, C4v orbits and the RDMFT lattice step.

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
    """

    def __init__(self, Lx, Ly=None, geometry=0, periodic=False, t=1.0, V0=0.0):
        self.geometry = geometry
        self.t = float(t)
        self.V0 = float(V0)
        if geometry == 0:
            Ly = Lx if Ly is None else Ly
            xs, ys = [], []
            for y in range(Ly):
                for x in range(Lx):
                    xs.append(x)
                    ys.append(y)
            self.x = np.array(xs)
            self.y = np.array(ys)
            self.cx, self.cy = (Lx - 1) / 2.0, (Ly - 1) / 2.0
            self.dx = self.x - self.cx
            self.dy = self.y - self.cy
        elif geometry == 1:
            R = Lx
            xs, ys = [], []
            for y in range(-R, R + 1):
                for x in range(-R, R + 1):
                    if x * x + y * y <= R * R:
                        xs.append(x)
                        ys.append(y)
            self.x = np.array(xs)
            self.y = np.array(ys)
            self.cx, self.cy = 0.0, 0.0
            self.dx = self.x.astype(float)
            self.dy = self.y.astype(float)
        else:
            raise ValueError("geometry")
        self.N = len(self.x)
        self.r2 = self.dx ** 2 + self.dy ** 2
        self.V = self.V0 * self.r2
        self.parity = np.where((self.x + self.y) % 2 == 0, 1, -1)
        index = {(int(a), int(b)): i for i, (a, b) in enumerate(zip(self.x, self.y))}
        A = np.zeros((self.N, self.N))
        for i in range(self.N):
            for (ddx, ddy) in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                xn, yn = int(self.x[i]) + ddx, int(self.y[i]) + ddy
                if periodic and geometry == 0:
                    xn %= Lx
                    yn %= Ly
                j = index.get((xn, yn))
                if j is not None and j != i:
                    A[i, j] = 1.0
        self.adjacency = A
        self.z = A.sum(axis=1)  # number of neighbours of each site
        self.H0 = -self.t * A + np.diag(self.V)
        self._index = index

    # --- C4v orbits -------------------------------------------------------
    def orbits(self):
        """Inequivalent sites under the point group of the trap and the lattice.

        The 8 operations (dx, dy) -> (+-dx, +-dy), (+-dy, +-dx) about the trap centre are kept if
        they map the site set onto itself.  Returns (reps, rep_of, flip): reps = sorted site
        indices of the orbit representatives; rep_of[i] = position in reps of the orbit of site i;
        flip[i] = 1 if site i and its representative lie on different sublattices.  An
        antiferromagnetic state then satisfies G_{i,sigma} = G_{rep, sigma xor flip}.
        """
        ops = []
        for swap in (False, True):
            for sx in (1, -1):
                for sy in (1, -1):
                    ops.append((swap, sx, sy))
        images = []
        for (swap, sx, sy) in ops:
            a = np.where(swap, self.dy, self.dx) * sx
            b = np.where(swap, self.dx, self.dy) * sy
            img = []
            ok = True
            for i in range(self.N):
                key = self._coord_to_index(a[i], b[i])
                if key is None:
                    ok = False
                    break
                img.append(key)
            if ok:
                images.append(np.array(img))
        rep_site = np.array([min(int(im[i]) for im in images) for i in range(self.N)])
        reps = np.array(sorted(set(rep_site.tolist())))
        pos = {int(r): k for k, r in enumerate(reps)}
        rep_of = np.array([pos[int(r)] for r in rep_site])
        flip = (self.parity != self.parity[rep_site]).astype(np.int64)
        return reps, rep_of, flip

    def _coord_to_index(self, ddx, ddy):
        x, y = ddx + self.cx, ddy + self.cy
        xi, yi = int(round(x)), int(round(y))
        if abs(x - xi) > 1e-9 or abs(y - yi) > 1e-9:
            return None
        return self._index.get((xi, yi))


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
