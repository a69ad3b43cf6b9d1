"""Entropy of the trapped system from densities ("Results for square lattice"): Monte Carlo
sampling gives no direct access to the entropy, so it is obtained from the thermodynamic relation
dS/dmu = dN/dT, integrating the temperature derivative of the density over the chemical potential
from an empty system (mu -> -infinity, S = 0).  The same relation, applied to the local density,
gives the entropy density of each site (the paper's "central site" curve).

This module drives the solver over the (T, mu) grid through the C ABI.  Each grid point is its own
RDMFT run (a context), and up to 8 of them go into one fused batch, so their impurity sweeps
share launches and their iterations replay from one CUDA graph.  Post-processing runs on the
host: a central difference in T and composite Simpson integration in mu.
"""
from __future__ import annotations

import numpy as np

from . import hf

_BATCH = 8


def density_scan(cfg: dict, temps, mus, L: int, iterations: int, device="cuda:0"):
    """Total density (both spins) of every inequivalent site after `iterations` RDMFT iterations
    at every (T, mu): returns (n [len(temps)][len(mus)][n_sites], multiplicity [n_sites]).

    cfg: a workload configuration (lattice, U, V0, sweeps, ...); beta = 1/T, dtau = beta/L, and
    mu are set per point.  Every run starts from the configuration's seeded self-energy."""
    import torch

    dev = torch.device(device)
    stream = torch.cuda.Stream(dev)
    points = [(a, b) for a in range(len(temps)) for b in range(len(mus))]
    _, ns, _, _, _, rep_of, _ = hf.hf_lattice_info(hf.make_params(cfg))
    mult = np.bincount(rep_of, minlength=ns).astype(np.float64)
    out = np.zeros((len(temps), len(mus), ns))
    for g0 in range(0, len(points), _BATCH):
        group = points[g0:g0 + _BATCH]
        ctxs = []
        for (a, b) in group:
            beta = 1.0 / float(temps[a])
            p = hf.make_params(dict(cfg, beta=beta, dtau=beta / L, mu=float(mus[b])))
            ctxs.append(hf.Context(p, device=dev, stream=stream))
        batch = hf.hf_batch_create([c.handle for c in ctxs], use_graph=1)
        try:
            for _ in range(iterations):
                hf.hf_batch_rdmft_step(batch)
        finally:
            hf.hf_batch_free(batch)
        for (a, b), c in zip(group, ctxs):
            mean, _ = hf.hf_get_observables(c.handle, ns, L)
            out[a, b] = mean[:, 2 * L] + mean[:, 2 * L + 1]
            c.close()
    return out, mult


def cumulative_simpson(mus, y):
    """Integral of y (last axis: the mu grid, uniform, odd length) from mus[0] up to each
    even-index point by composite Simpson; returns values at mus[0::2]."""
    mus = np.asarray(mus, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m = len(mus)
    if m < 3 or m % 2 == 0:
        raise ValueError("Simpson integration needs an odd number (>= 3) of mu points")
    h = mus[1] - mus[0]
    if not np.allclose(np.diff(mus), h, rtol=1e-9, atol=1e-12):
        raise ValueError("the mu grid must be uniform")
    panels = (h / 3.0) * (y[..., 0:m - 2:2] + 4.0 * y[..., 1:m - 1:2] + y[..., 2:m:2])
    zero = np.zeros(y.shape[:-1] + (1,))
    return np.concatenate([zero, np.cumsum(panels, axis=-1)], axis=-1)


def entropy_scan(cfg: dict, T: float, dT: float, mus, L: int, iterations: int, device="cuda:0"):
    """Entropy at temperature T on the chemical-potential grid `mus` (uniform, odd length, its
    first point deep enough that the trap is empty): S(mu) - S(mus[0]) = integral of dN/dT, with
    dN/dT from densities at T - dT and T + dT.

    Returns a dict with mu (mus[0::2]), S (total), s_site (per inequivalent site), N (density sum
    at T, the mean of the two temperatures), n_site, dn_dT (per site, every mu)."""
    n, mult = density_scan(cfg, (T - dT, T + dT), mus, L, iterations, device=device)
    dn_dT = (n[1] - n[0]) / (2.0 * dT)                     # [mu][site]
    s_site = cumulative_simpson(mus, dn_dT.T)               # [site][mu/2]
    S = mult @ s_site
    n_mid = 0.5 * (n[0] + n[1])
    return {"mu": np.asarray(mus)[0::2], "S": S, "s_site": s_site, "N": n_mid @ mult,
            "n_site": n_mid, "dn_dT": dn_dT, "multiplicity": mult}
