"""Kirkwood's solution for point charges inside a dielectric sphere in a linear ionic solvent.

TEST INFRASTRUCTURE. Used as the analytic reference of Section 3.1 (the Kirkwood sphere).

The reaction field is obtained by matching Legendre modes at r = a: inside the sphere the
potential is sum_k q_k/(eps1 |r - r_k|) + sum_n A_n r^n P_n, outside it is
sum_n B_n k_n(kappa r) P_n with k_n the modified spherical Bessel function of the second
kind. Continuity of the potential and of eps * d(phi)/dr (eqJump) give, per source charge,

    A_n = q r_k^n (eps1 (n+1) + g_n) / (eps1 a^(2n+1) (eps1 n - g_n)),
    g_n = eps2 x k_n'(x)/k_n(x),  x = kappa a,

and E = 1/2 sum_j q_j phi_reac(r_j) (solvation_energy), times 332.0716 for kcal/mol.
The ratio x k_n'/k_n = -x k_{n-1}/k_n - (n+1) is evaluated with the three-term recurrence
k_{n+1} = k_{n-1} + (2n+1)/x k_n, carried as the ratio k_{n-1}/k_n, which never overflows.

Pins (tests/test_oracle_kirkwood.py): the n = 0 term alone equals the closed form for a
centred charge; kappa = 0 reproduces the Born-Kirkwood factor
(n+1)(eps1-eps2)/(eps1(n eps1 + (n+1) eps2)); the printed exact energy -8273.31 kcal/mol of
Table 1 is reproduced for a = 50, q = 50, eps2/eps1 = 40 at kappa = 0.1257.
"""
from __future__ import annotations

import numpy as np

COULOMB = 332.0716


def centered(q, a, eps1, eps2, kappa):
    """Closed-form solvation energy (kcal/mol) of one charge at the centre of the sphere."""
    return COULOMB * q * q / (2.0 * a) * (1.0 / (eps2 * (1.0 + kappa * a)) - 1.0 / eps1)


def _g(nmax, x, eps2):
    """g_n = eps2 x k_n'(x)/k_n(x) for n = 0..nmax."""
    g = np.zeros(nmax + 1)
    g[0] = eps2 * (-x - 1.0)
    if x == 0.0:
        for n in range(nmax + 1):
            g[n] = -(n + 1) * eps2
        return g
    rho = x / (1.0 + x)  # k_0/k_1
    for n in range(1, nmax + 1):
        g[n] = eps2 * (-x * rho - (n + 1))
        rho = 1.0 / (rho + (2 * n + 1) / x)  # k_n/k_{n+1}
    return g


def _legendre(nmax, t):
    P = np.zeros(nmax + 1)
    P[0] = 1.0
    if nmax >= 1:
        P[1] = t
    for n in range(1, nmax):
        P[n + 1] = ((2 * n + 1) * t * P[n] - n * P[n - 1]) / (n + 1)
    return P


def series(qpos, q, a, eps1, eps2, kappa, center=(0.0, 0.0, 0.0), tol=1e-17, nmax=2000):
    """Solvation energy (kcal/mol) of charges q at qpos inside a sphere of radius a."""
    qpos = np.asarray(qpos, dtype=np.float64).reshape(-1, 3) - np.asarray(center)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    r = np.linalg.norm(qpos, axis=1)
    if np.any(r >= a):
        raise ValueError("charges must lie strictly inside the sphere")
    rmax = r.max() if r.size else 0.0
    ratio = (rmax / a) ** 2
    if ratio <= 0.0:
        n_needed = 1
    else:
        n_needed = int(min(nmax, max(1, np.ceil(np.log(tol) / np.log(ratio)) + 1)))
    g = _g(n_needed, kappa * a, eps2)
    n = np.arange(n_needed + 1)
    fac = (eps1 * (n + 1) + g) / (eps1 * n - g) / (eps1 * a ** (2 * n + 1))
    E = 0.0
    for j in range(q.size):
        for k in range(q.size):
            rr = r[j] * r[k]
            if rr == 0.0:
                cosg = 1.0
            else:
                cosg = float(np.clip(qpos[j] @ qpos[k] / rr, -1.0, 1.0))
            P = _legendre(n_needed, cosg)
            E += q[j] * q[k] * np.sum(rr ** n * P * fac)
    return 0.5 * COULOMB * E


def surface_fields_centered(q, a, eps1, eps2, kappa):
    """Exact surface potential phi_1 and its normal derivative for a centred charge, in the
    paper's units e_c/(4 pi Angstrom) (G0 = 1/(4 pi r), S1 = q G0/eps1)."""
    phi = q / (4.0 * np.pi * eps2 * (1.0 + kappa * a) * a)
    dphi = -q / (4.0 * np.pi * eps1 * a * a)
    return phi, dphi
