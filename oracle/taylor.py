"""Taylor coefficients of the Coulomb and screened Coulomb kernels by power-series arithmetic.

TEST INFRASTRUCTURE. The Cartesian FMM of Section 2.4 needs the derivatives D^gamma G of
G0 = 1/(4 pi r) and Gk = exp(-kappa r)/(4 pi r) at the vector between two cluster centres
(eqcoeff). The paper cites a recurrence for them; this module obtains the same numbers by a
different route, so that it can pin the CUDA recurrence: truncated multivariate power series
in h = (h1, h2, h3), composed step by step,

    r^2(d + h) = |d|^2 + 2 d.h + |h|^2,
    1/r        = sum_n binom(-1/2, n) |d|^(-1-2n) (r^2 - |d|^2)^n,
    r          = sum_n binom(1/2, n)  |d|^(1-2n)  (r^2 - |d|^2)^n,
    exp(-k r)  = exp(-k |d|) sum_n (-k (r - |d|))^n / n!,

each truncated at total degree p. The coefficient of h^gamma is D^gamma G(d)/gamma!.

Pins (tests/test_oracle_taylor_fmm.py): degree-0 and degree-1 coefficients equal the closed forms
G(d) and grad G(d); second-order coefficients equal the Hessian; all coefficients to |gamma|
= 6 agree with central finite differences of the closed form; Gk at kappa = 0 equals G0;
G0 satisfies Laplace's equation coefficient-wise.
"""
from __future__ import annotations

from math import factorial

import numpy as np


def multi_indices(p):
    """All (a, b, c) with a + b + c <= p, ordered by total degree, then a descending, then b
    descending. This order is the layout of every moment and local-expansion vector."""
    out = []
    for n in range(p + 1):
        for a in range(n, -1, -1):
            for b in range(n - a, -1, -1):
                out.append((a, b, n - a - b))
    return out


def nterms(p):
    return (p + 1) * (p + 2) * (p + 3) // 6


class Series:
    """Batch of truncated power series in three variables: array (..., p+1, p+1, p+1), zero
    above total degree p. The leading axes index independent series (one per cluster pair)."""

    def __init__(self, p, c):
        self.p = p
        self.c = c

    @staticmethod
    def const(p, batch, value):
        c = np.zeros(tuple(batch) + (p + 1,) * 3)
        c[..., 0, 0, 0] = value
        return Series(p, c)

    def __add__(self, o):
        if isinstance(o, Series):
            return Series(self.p, self.c + o.c)
        c = self.c.copy()
        c[..., 0, 0, 0] += o
        return Series(self.p, c)

    def scale(self, v):
        """multiply by a scalar or a per-series array v (shape = batch)"""
        v = np.asarray(v, dtype=np.float64)
        return Series(self.p, self.c * v[..., None, None, None])

    def __mul__(self, o):
        p = self.p
        out = np.zeros_like(self.c)
        for a, b, c in multi_indices(p):
            v = self.c[..., a, b, c]
            if not np.any(v):
                continue
            v = v[..., None, None, None]
            out[..., a:, b:, c:] += v * o.c[..., : p + 1 - a, : p + 1 - b, : p + 1 - c]
        i, j, k = np.indices((p + 1,) * 3)
        out[..., i + j + k > p] = 0.0
        return Series(p, out)


def _compose(delta, coeffs):
    """sum_n coeffs[n] delta^n for series delta with zero constant term; coeffs[n] has the
    batch shape."""
    p = delta.p
    batch = delta.c.shape[:-3]
    out = Series.const(p, batch, 0.0)
    term = Series.const(p, batch, 1.0)
    for n in range(p + 1):
        out = out + term.scale(coeffs[n])
        if n < p:
            term = delta * term
    return out


def _binom(alpha, n):
    r = 1.0
    for k in range(n):
        r *= (alpha - k) / (k + 1)
    return r


def kernel_series(d, p, kappa):
    """Series of G0 (kappa = 0) or Gk about each row of d (shape (..., 3)); coefficient
    [..., a, b, c] = D^(a,b,c) G(d)/(a! b! c!)."""
    d = np.asarray(d, dtype=np.float64)
    batch = d.shape[:-1]
    u0 = np.einsum("...k,...k->...", d, d)
    r0 = np.sqrt(u0)
    c = np.zeros(tuple(batch) + (p + 1,) * 3)
    # r^2 - |d|^2 = 2 d.h + |h|^2
    if p >= 1:
        c[..., 1, 0, 0] = 2 * d[..., 0]
        c[..., 0, 1, 0] = 2 * d[..., 1]
        c[..., 0, 0, 1] = 2 * d[..., 2]
    if p >= 2:
        c[..., 2, 0, 0] = 1.0
        c[..., 0, 2, 0] = 1.0
        c[..., 0, 0, 2] = 1.0
    delta = Series(p, c)
    inv_r = _compose(delta, [_binom(-0.5, n) * u0 ** (-0.5 - n) for n in range(p + 1)])
    G = inv_r.scale(1.0 / (4.0 * np.pi))
    if kappa == 0.0:
        return G
    r = _compose(delta, [_binom(0.5, n) * u0 ** (0.5 - n) for n in range(p + 1)])
    rho = Series(p, r.c.copy())
    rho.c[..., 0, 0, 0] = 0.0
    ex = _compose(rho, [np.exp(-kappa * r0) * (-kappa) ** n / factorial(n) for n in range(p + 1)])
    return ex * G


def derivatives(d, p, kappa):
    """D^gamma G(d) for all |gamma| <= p, last axis in multi_indices(p) order."""
    s = kernel_series(d, p, kappa)
    idx = multi_indices(p)
    fac = np.array([factorial(a) * factorial(b) * factorial(c) for a, b, c in idx], dtype=np.float64)
    a = np.array([t[0] for t in idx])
    b = np.array([t[1] for t in idx])
    cc = np.array([t[2] for t in idx])
    return s.c[..., a, b, cc] * fac
