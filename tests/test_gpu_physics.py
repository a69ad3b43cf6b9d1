"""Physics cross-check with the parameters of the paper's Fig. 1 (square lattice, V0 = 0.25,
U = 10, dtau = 0.1), qualitative as the paper's own statements are: at low temperature a large
antiferromagnetic core polarised up to ~90%, no order above T_N ~ 0.32, a double occupancy of
about 0.02 at the centre at high temperature that the ordered core enhances by up to ~50%, and a
density profile that hardly changes with temperature.

A site-centred 17x17 trap, half filled at its centre (mu = U/2), 16 chains per inequivalent site,
20 RDMFT iterations (mixing 0.5 from the staggered seed field) at T = 0.156 (L = 64) and T = 0.5
(L = 20).  The margins are wide: this checks the physics, not parity (parity is checked against
the oracle elsewhere).
"""
import numpy as np
import pytest

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


def _run(hf, T, L):
    import torch

    cfg = dict(wl.CONFIGS["square20"], Lx=17, Ly=17, U=10.0, V0=0.25, mu=5.0, dtau=0.1,
               beta=1.0 / T, chains_per_site=16, precision=2, h_seed=0.1, mix=0.5)
    ctx = hf.Context(hf.make_params(cfg), stream=torch.cuda.Stream())
    for _ in range(20):
        hf.hf_rdmft_step(ctx.handle)
    rep, _, _ = hf.hf_get_orbits(ctx.handle, ctx.n_sites, ctx.N)
    mean, _ = hf.hf_get_observables(ctx.handle, ctx.n_sites, L)
    ctx.close()
    x, y = rep % 17 - 8, rep // 17 - 8
    parity = np.where((x + y) % 2 == 0, 1.0, -1.0)
    n = mean[:, 2 * L] + mean[:, 2 * L + 1]
    return np.hypot(x, y), n, mean[:, 2 * L + 2], mean[:, 2 * L + 3] * parity


def test_fig1_melting_of_the_af_core(hf):
    r, n_lo, d_lo, m_lo = _run(hf, 0.15625, 64)
    _, n_hi, d_hi, m_hi = _run(hf, 0.5, 20)
    c = int(np.argmin(r))
    core = r <= 3.0
    assert abs(n_lo[c] - 1.0) < 0.02                       # half filled at the centre
    assert abs(m_lo[c]) / n_lo[c] > 0.8                    # strongly polarised core at low T
    assert np.all(np.abs(m_lo[core]) > 0.5)
    assert abs(m_hi[c]) / n_hi[c] < 0.1                    # paramagnetic above T_N
    assert 0.015 < d_hi[c] < 0.035                         # ~0.02 at the centre at high T
    ratio = d_lo[core].mean() / d_hi[core].mean()
    assert 1.2 < ratio < 1.8                               # enhanced by up to ~50% in the core
    assert np.abs(n_lo - n_hi).max() < 0.1                 # density nearly unchanged
