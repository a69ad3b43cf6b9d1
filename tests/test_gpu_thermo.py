"""The entropy scan (dS/dmu = dN/dT integrated from the empty trap, "Results for square lattice")
through the C ABI on the GPU, pinned at U = 0, where the RDMFT solution is the free lattice
(Sigma = 0) and the entropy has a closed form (oracle/thermo.py).

Grid: T = 0.5 with T +- 0.01, mu from -10 (trap empty to e^-12) to 0 in steps of 0.25 (41 points,
82 RDMFT runs in fused batches of 8).  The discretisation alone -- the central difference in T and
Simpson's rule in mu, applied to exact densities -- is within 2.4e-5 of the exact entropy for this
grid, so the bar is 1e-4 relative for the total entropy and 1e-4 absolute per site.
"""
import numpy as np
import pytest

from oracle import thermo as ot
from oracle.lattice import Lattice
from paper_1006_2716_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1006_2716_gb300 import build as B

    B.build()
    from paper_1006_2716_gb300 import hf as H

    return H


def test_entropy_scan_free_trap(hf):
    from paper_1006_2716_gb300 import thermo

    cfg = dict(wl.CONFIGS["square6"], U=0.0, h_seed=0.0, precision=2, chains_per_site=1,
               n_warmup=0, n_measure=1, bin_size=1, max_bins=1)
    T, dT = 0.5, 0.01
    mus = np.linspace(-10.0, 0.0, 41)
    res = thermo.entropy_scan(cfg, T, dT, mus, L=8, iterations=1)
    lat = Lattice(6, 6, V0=cfg["V0"])
    reps, rep_of, _ = lat.orbits()
    s_exact = np.array([ot.free_entropy(lat.H0, m, T) - ot.free_entropy(lat.H0, mus[0], T)
                        for m in res["mu"]])                     # [mu/2][site]
    S_exact = s_exact.sum(axis=1)
    assert np.abs(res["S"] - S_exact).max() < 1e-4 * S_exact[-1]
    assert np.abs(res["s_site"].T - s_exact[:, reps]).max() < 1e-4
    # the densities themselves: the free lattice at T -+ dT
    n_exact = 0.5 * (ot.free_density(lat.H0, mus[-1], T - dT) + ot.free_density(lat.H0, mus[-1], T + dT))
    assert np.abs(res["n_site"][-1] - n_exact[reps]).max() < 1e-8
    assert abs(res["N"][-1] - n_exact.sum()) < 1e-7
    assert np.array_equal(res["multiplicity"], np.bincount(rep_of).astype(float))
