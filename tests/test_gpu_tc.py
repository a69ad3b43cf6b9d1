"""The tensor-core building blocks of the L = 128 refresh.

* hf_tc_dgemm128 (exact-digit products on tcgen05): operands that one digit represents exactly
  give the exact product bit for bit, which pins the shared-memory operand layout, the MMA
  descriptors and the TMEM read-back; general FP64 operands with 3, 5 and 7 digits stay within
  the error bound of the dropped digits and levels, measured against a 113-bit (or 64-bit)
  long-double product.
* The refresh of the mixed-precision form: after FP32 sweeps, the FP64 G that the Newton steps
  on the tensor cores produce gives the measurement of the exact Dyson solution (the oracle's,
  refined in long double) within 1e-12 of G's largest entry; a chain whose FP32 state is far from
  its inverse, or whose G is too badly conditioned for the residual's fixed-point accuracy, falls
  back to Gauss-Jordan and still gives the oracle's answer.
"""
import numpy as np
import pytest

import oracle as o
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


def _dgemm(hf, A, B, digits):
    import torch

    n = A.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    dC = torch.full((n, 128, 128), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    hf.hf_tc_dgemm128(dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), n, digits, st.data_ptr())
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return dC.cpu().numpy()


def _scales(X, axis):
    m = np.abs(X).max(axis=axis)
    return np.floor(np.log2(m)) + 2


def test_one_digit_operands_give_the_exact_product(hf):
    rng = np.random.default_rng(1)
    n = 3
    # integers in [-127, 127] with a row (column) maximum in [64, 127] are one exact digit
    Ai = rng.integers(-127, 128, size=(n, 128, 128))
    Bi = rng.integers(-127, 128, size=(n, 128, 128))
    Ai[:, :, 0] = 100
    Bi[:, 0, :] = -90
    A = Ai * 2.0 ** rng.integers(-6, 6, size=(n, 128, 1))     # power-of-two row scales
    B = Bi * 2.0 ** rng.integers(-6, 6, size=(n, 1, 128))     # and column scales
    C = _dgemm(hf, A, B, 1)
    want = np.einsum("bik,bkj->bij", A, B)                     # exact: integer sums < 2^53
    assert np.array_equal(C, want)


@pytest.mark.parametrize("digits", [3, 5, 7, 8])
def test_digit_products_within_their_bound(hf, digits):
    rng = np.random.default_rng(digits)
    n = 4
    A = rng.standard_normal((n, 128, 128)) * np.exp(rng.uniform(-3, 3, (n, 128, 1)))
    B = rng.standard_normal((n, 128, 128)) * np.exp(rng.uniform(-3, 3, (n, 1, 128)))
    C = _dgemm(hf, A, B, digits)
    Al, Bl = A.astype(np.longdouble), B.astype(np.longdouble)
    for b in range(n):
        exact = Al[b] @ Bl[b]
        scale = 2.0 ** (_scales(A[b], 1)[:, None] + _scales(B[b], 0)[None, :])
        err = np.abs((C[b] - exact).astype(np.float64)) / scale
        # dropped digits and levels: below 2^(9 - 8 digits) of the scales (8 digits: the 62-bit
        # fixed-point operands exactly); from 7 digits on, the FP64 rounding of C itself (|C_ij| up
        # to 2^(TA_i + TB_j + 5)) dominates
        assert err.max() < 2.0 ** (max(9 - 8 * digits, -46)), (digits, err.max())
    if digits >= 7:   # and as good as a plain FP64 product relative to |A||B|
        ref = np.abs(A[0]) @ np.abs(B[0])
        assert (np.abs(C[0] - (Al[0] @ Bl[0]).astype(np.float64)) / ref).max() < 1e-14


def test_rejects_bad_arguments(hf):
    import torch

    buf = torch.zeros(128 * 128, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    for args in ((p, p, p, 1, 4), (p, p, p, -1, 7), (p + 8, p, p, 1, 7)):
        with pytest.raises(hf.HFError):
            hf.hf_tc_dgemm128(*args)
    hf.hf_tc_dgemm128(p, p, p, 0, 7)


def _ctx(hf, **over):
    cfg = dict(wl.CONFIGS["square6"], precision=1, refresh_every=1, beta=16.0, dtau=0.125,
               U=8.0, bin_size=1, max_bins=1)
    cfg.update(over)
    return hf.Context(hf.make_params(cfg)), cfg


def _exact_dyson(g0, s, sigma, lam):
    """The Dyson solution G = A^{-1} g0 to (nearly) full FP64 accuracy: the oracle's elimination
    result, refined twice with residuals g0 - A G formed in long double (classical iterative
    refinement; the elimination's own error grows with the conditioning of A)."""
    G, _ = o.dyson(g0, s, sigma, lam)
    L = g0.shape[0]
    ev = np.exp(lam * sigma * s.astype(np.float64)) - 1.0
    A = np.eye(L) + (np.eye(L) - g0) * ev[None, :]
    Al = np.eye(L, dtype=np.longdouble) + (np.eye(L, dtype=np.longdouble) - g0.astype(np.longdouble)) \
        * np.expm1(np.longdouble(lam) * sigma * s.astype(np.longdouble))[None, :]
    for _ in range(2):
        r = (g0.astype(np.longdouble) - Al @ G.astype(np.longdouble)).astype(np.float64)
        G = G + np.linalg.solve(A, r)
    return G


def _set_baths(hf, ctx, baths):
    for i in range(ctx.n_sites):
        for sp in range(2):
            hf.hf_set_g0(ctx.handle, i, sp, baths[i, sp])


@pytest.mark.parametrize("U,seed", [(8.0, 5), (4.0, 6), (10.0, 7)])
def test_tensor_core_refresh_matches_oracle_dyson(hf, U, seed):
    L = 128
    ctx, cfg = _ctx(hf, chains_per_site=2, U=U, seed=seed)
    gj, _ = _ctx(hf, chains_per_site=2, U=U, seed=seed, refresh_gj=1)
    baths = wl.random_baths(seed + 40, ctx.n_sites, cfg["beta"], L)
    for c in (ctx, gj):
        _set_baths(hf, c, baths)
        hf.hf_sweep(c.handle, 3, 1, 1)       # 3 sweeps + refreshes, then 1 measured
    f, _ = hf.hf_get_fields(ctx.handle, ctx.n_chains, L)
    fg, _ = hf.hf_get_fields(gj.handle, gj.n_chains, L)
    tcn, fb, npr = hf.hf_get_refresh_stats(ctx.handle)
    print("\nU=%g: %d tensor-core chain refreshes, %d handed to Gauss-Jordan, %.1f digit products "
          "per refresh" % (U, tcn, fb, npr / max(tcn + fb, 1)))
    assert tcn + fb == 4 * ctx.n_chains and tcn > 0
    _, lam = o.constants(cfg["beta"], U, L)
    worst_tc, worst_gj = 0.0, 0.0
    for i in range(ctx.n_sites):
        g0u, g0d = o.build_g0(baths[i, 0]), o.build_g0(baths[i, 1])
        ref = np.zeros(2 * L + 3)
        scale = 0.0
        for ch in range(2):
            c = 2 * i + ch
            Gu = _exact_dyson(g0u, f[c], 1, lam)
            Gd = _exact_dyson(g0d, f[c], -1, lam)
            ref += o.measure(Gu, Gd) / 2
            scale = max(scale, np.abs(Gu).max(), np.abs(Gd).max())
        gtau, n, d, m, _ = hf.hf_measure(ctx.handle, i, L)
        got = np.concatenate([gtau, n, [d]])
        worst_tc = max(worst_tc, np.abs(got - ref).max() / scale)
        if np.array_equal(f[2 * i:2 * i + 2], fg[2 * i:2 * i + 2]):
            g2 = hf.hf_measure(gj.handle, i, L)
            worst_gj = max(worst_gj, np.abs(np.concatenate([g2[0], g2[1], [g2[2]]]) - ref).max() / scale)
    print("max |measurement - exact Dyson| / max|G|: tensor-core %.2e, Gauss-Jordan %.2e"
          % (worst_tc, worst_gj))
    # relative to G's largest entry, as the FP64 refresh is judged elsewhere (1e-10 there)
    assert worst_tc < 1e-12
    ctx.close()
    gj.close()


def test_far_state_falls_back_to_gauss_jordan(hf):
    """Fields replaced without a refresh leave an FP32 state that is no approximate inverse of the
    new M: the Newton residual does not converge, the chain is refreshed by Gauss-Jordan, and the
    measurement after the sweep is still the oracle's Dyson answer for the fields it ends with."""
    L = 128
    ctx, cfg = _ctx(hf, chains_per_site=1, U=8.0, seed=9, Lx=2, Ly=2)
    baths = wl.random_baths(77, ctx.n_sites, cfg["beta"], L)
    _set_baths(hf, ctx, baths)
    hf.hf_sweep(ctx.handle, 2, 0, 1)
    f, cnt = hf.hf_get_fields(ctx.handle, ctx.n_chains, L)
    rng = np.random.default_rng(3)
    f2 = np.where(rng.random(f.shape) < 0.5, 1, -1).astype(np.int8)
    hf.hf_set_fields(ctx.handle, f2, cnt)
    hf.hf_clear_measurements(ctx.handle)
    hf.hf_sweep(ctx.handle, 0, 1, 0)          # no refresh first: the sweep starts from the old G
    f3, _ = hf.hf_get_fields(ctx.handle, ctx.n_chains, L)
    tcn, fb, _ = hf.hf_get_refresh_stats(ctx.handle)
    assert fb == ctx.n_chains and tcn == 0, (tcn, fb)
    _, lam = o.constants(cfg["beta"], 8.0, L)
    for i in range(ctx.n_sites):
        Gu, _ = o.dyson(o.build_g0(baths[i, 0]), f3[i], 1, lam)
        Gd, _ = o.dyson(o.build_g0(baths[i, 1]), f3[i], -1, lam)
        ref = o.measure(Gu, Gd)
        gtau, n, d, m, _ = hf.hf_measure(ctx.handle, i, L)
        assert np.abs(gtau - ref[:2 * L]).max() < 1e-10
        assert abs(d - ref[2 * L + 2]) < 1e-10
    ctx.close()
