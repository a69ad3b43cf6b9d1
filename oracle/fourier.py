"""Imaginary-time <-> Matsubara transforms of the oracle (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper keeps 500 Matsubara frequencies explicitly ("Model and Methods", eq. 2 paragraph) and
couples them through the impurity problem, but does not write the transforms down.  The readings
used here:

* Physics convention G(i w) = int_0^beta e^{i w tau} G(tau) dtau, G(tau) = -<T c(tau) c^+>;
  the oracle reports the positive g(tau) = -G(tau), so g(0+) = 1 - n, g(beta-) = n.
* i w -> tau: g(tau) = -2T sum_{n<nw} Re[e^{-i w_n tau}(G(i w_n) - tail(i w_n))] + g_tail(tau)
  with tail = 1/(i w) + c2/(i w)^2 + c3/(i w)^3 whose positive-convention images are
  1/2, c2 (beta - 2 tau)/4 and -c3 tau (beta - tau)/4 on 0 < tau < beta.
* tau -> i w: G(i w) = G_ref(i w) + FT[spline(g - g_ref)], natural cubic spline through the
  L + 1 points tau_m = m dtau (m = L is beta-), integrated exactly segment by segment.
"""
from __future__ import annotations

import numpy as np


def matsubara(beta, nw):
    return (2.0 * np.arange(nw) + 1.0) * np.pi / beta


def tail(iw, c2, c3):
    return 1.0 / iw + c2 / iw ** 2 + c3 / iw ** 3


def iw_to_tau(beta, G_iw, c2, c3, L):
    """Positive-convention g(tau_m), m = 0..L (tau_0 = 0+, tau_L = beta-), of one G(i w_n)."""
    nw = G_iw.shape[0]
    w = matsubara(beta, nw)
    iw = 1j * w
    rem = G_iw - tail(iw, c2, c3)
    out = np.zeros(L + 1)
    for m in range(L + 1):
        tau = beta * m / L
        s = np.sum(np.real(np.exp(-1j * w * tau) * rem))
        g = -(2.0 / beta) * s
        g += 0.5 + c2 * (beta - 2.0 * tau) / 4.0 - c3 * tau * (beta - tau) / 4.0
        out[m] = g
    return out


def natural_spline_coeffs(h, y):
    """Piecewise cubic a + b x + c x^2 + d x^3 (x from the left knot) through y on a uniform
    grid of spacing h, second derivative zero at both ends.  Returns arrays a, b, c, d."""
    n = y.shape[0] - 1  # segments
    M = np.zeros(n + 1)
    if n >= 2:
        A = np.zeros((n - 1, n - 1))
        rhs = np.zeros(n - 1)
        for k in range(1, n):
            A[k - 1, k - 1] = 4.0
            if k - 2 >= 0:
                A[k - 1, k - 2] = 1.0
            if k < n - 1:
                A[k - 1, k] = 1.0
            rhs[k - 1] = 6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]) / h ** 2
        M[1:n] = np.linalg.solve(A, rhs)
    a = y[:-1].copy()
    b = (y[1:] - y[:-1]) / h - h * (2.0 * M[:-1] + M[1:]) / 6.0
    c = M[:-1] / 2.0
    d = (M[1:] - M[:-1]) / (6.0 * h)
    return a, b, c, d


def spline_fourier(beta, dg, nw):
    """Physics-convention Fourier integral int_0^beta e^{i w_n tau} (-spline(dg))(tau) dtau.

    dg: positive-convention values at tau_m = m beta / L, m = 0..L.
    """
    L = dg.shape[0] - 1
    h = beta / L
    a, b, c, d = natural_spline_coeffs(h, dg)
    w = matsubara(beta, nw)
    iw = 1j * w
    out = np.zeros(nw, dtype=np.complex128)
    for m in range(L):
        t0 = m * h
        # p(x) = a + b x + c x^2 + d x^3 on [0, h]; int_0^h e^{iwx} p(x) dx by parts
        p = [a[m], b[m], c[m], d[m]]

        def deriv(k, x):
            if k == 0:
                return p[0] + p[1] * x + p[2] * x ** 2 + p[3] * x ** 3
            if k == 1:
                return p[1] + 2.0 * p[2] * x + 3.0 * p[3] * x ** 2
            if k == 2:
                return 2.0 * p[2] + 6.0 * p[3] * x
            return 6.0 * p[3]

        seg = np.zeros(nw, dtype=np.complex128)
        for k in range(4):
            term = (np.exp(iw * h) * deriv(k, h) - deriv(k, 0.0)) / iw ** (k + 1)
            seg += ((-1.0) ** k) * term
        out += np.exp(iw * t0) * seg
    return -out


def tau_to_iw(beta, g_tau, g_ref_tau, G_ref_iw):
    """G(i w) = G_ref(i w) + FT[spline(g - g_ref)] from g(tau_m), m = 0..L-1 (tau_0 = 0+).

    The beta- point is fixed by g(beta-) = 1 - g(0+) for both functions, so the difference
    there is -(g(0+) - g_ref(0+)).
    """
    L = g_tau.shape[0]
    dg = np.zeros(L + 1)
    dg[:L] = g_tau - g_ref_tau
    dg[L] = -dg[0]
    return G_ref_iw + spline_fourier(beta, dg, G_ref_iw.shape[0])
