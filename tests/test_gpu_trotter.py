"""Trotter extrapolation through the CUDA path: one impurity at dtau = beta / L for five L in one
fused uneven-L launch; the double occupancy, fitted as a + b dtau^2 with the measured errors,
extrapolates to the exact-diagonalisation value of the continuous-time impurity, and at the
smallest L it equals the exact discretised (brute-force) value."""
import numpy as np
import pytest

import oracle as o
from oracle.ed import anderson_ed
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


@pytest.mark.parametrize("precision", [2, 0])
def test_double_occupancy_extrapolates_to_exact(hf, precision):
    import torch

    beta, U, seed = 2.0, 2.0, 3
    e, w = wl.bath_poles(seed)
    _, _, d_ed = anderson_ed(e, w, U, beta, 8)
    Ls = [16, 24, 32, 48, 64]
    stream = torch.cuda.Stream()
    ctxs = []
    for k, L in enumerate(Ls):
        cfg = dict(wl.CONFIGS["square6"], Lx=1, Ly=1, beta=beta, dtau=beta / L, U=U, mu=0.0,
                   V0=0.0, precision=precision, chains_per_site=2048, n_matsubara=4,
                   refresh_every=10, bin_size=100, max_bins=20, seed=900 + k)
        ctx = hf.Context(hf.make_params(cfg), stream=stream)
        assert ctx.L == L
        bath = wl.pole_bath_tau(beta, L, e, w)
        hf.hf_set_g0(ctx.handle, 0, 0, bath)
        hf.hf_set_g0(ctx.handle, 0, 1, bath)
        ctxs.append(ctx)
    b = hf.hf_batch_create([c.handle for c in ctxs], 0)
    hf.hf_batch_sweep(b, 200, 2000, 1)
    d, sd = [], []
    for ctx, L in zip(ctxs, Ls):
        _, _, dd, _, errs = hf.hf_measure(ctx.handle, 0, L)
        d.append(dd)
        sd.append(errs[2 * L + 2])
    hf.hf_batch_free(b)
    for c in ctxs:
        c.close()
    d, sd = np.array(d), np.array(sd)
    dt = beta / np.array(Ls, dtype=float)
    # the smallest L against the exact discretised answer (all 2^16 fields)
    g0 = o.build_g0(wl.pole_bath_tau(beta, 16, e, w))
    _, lam = o.constants(beta, U, 16)
    d16 = o.brute_force(lam, g0, g0)[2 * 16 + 2]
    assert abs(d[0] - d16) < 4 * sd[0], (d[0], d16, sd[0])
    # weighted least squares a + b dtau^2
    A = np.stack([np.ones_like(dt), dt ** 2], axis=1) / sd[:, None]
    coef, *_ = np.linalg.lstsq(A, d / sd, rcond=None)
    cov = np.linalg.inv(A.T @ A)
    sa = np.sqrt(cov[0, 0])
    assert abs(d[0] - d_ed) > 4 * sd[0]            # the discretisation error is resolved ...
    assert abs(coef[0] - d_ed) < 4 * sa + 2e-5, (coef[0], d_ed, sa)   # ... and extrapolates away
