"""Pins of the dense Galerkin oracle (quadrature, pair integrals, assembly) against facts
that do not come from the oracle itself: exactness on polynomials, closed-form solid angles
of flat triangles (Van Oosterom-Strackee), brute-force refined quadrature, symmetries of the
kernels and the null case. CPU only."""
import itertools

import numpy as np
import pytest

from oracle import dense
from paper_2110_13778_gb300 import inputs


def _mono_exact(a, b):
    # int over {0 <= e2 <= e1 <= 1} of e1^a e2^b
    return 1.0 / ((b + 1) * (a + b + 2))


def test_gauss_legendre_exact_on_polynomials():
    for n in (1, 2, 3, 4, 6, 8):
        x, w = dense.gauss_legendre01(n)
        for k in range(2 * n):
            assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14


@pytest.mark.parametrize("case", [1, 2, 3])
def test_sauter_schwab_maps_integrate_polynomials(case):
    # The sub-maps must decompose tau x tau: every monomial in (xhat, yhat) integrates exactly.
    gx, gw = dense.gauss_legendre01(6)
    pts = []
    for i, j, k, l in itertools.product(range(6), repeat=4):
        xh, yh, jac = dense.ss_points(case, gx[i], gx[j], gx[k], gx[l])
        w = gw[i] * gw[j] * gw[k] * gw[l]
        for s in range(len(jac)):
            pts.append((xh[s, 0], xh[s, 1], yh[s, 0], yh[s, 1], w * jac[s]))
    P = np.array(pts)
    for a, b, c, d in itertools.product(range(3), repeat=4):
        got = np.sum(P[:, 4] * P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** c * P[:, 3] ** d)
        ref = _mono_exact(a, b) * _mono_exact(c, d)
        assert abs(got - ref) < 1e-13 * max(1.0, ref), (a, b, c, d)


def _solid_angle(x, P):
    """Signed solid angle of triangle P seen from points x (Van Oosterom & Strackee 1983)."""
    R = P[None, :, :] - x[:, None, :]
    r = np.linalg.norm(R, axis=2)
    num = np.einsum("ij,ij->i", R[:, 0], np.cross(R[:, 1], R[:, 2]))
    den = (r[:, 0] * r[:, 1] * r[:, 2] + np.einsum("ij,ij->i", R[:, 0], R[:, 1]) * r[:, 2]
           + np.einsum("ij,ij->i", R[:, 0], R[:, 2]) * r[:, 1] + np.einsum("ij,ij->i", R[:, 1], R[:, 2]) * r[:, 0])
    return 2.0 * np.arctan2(num, den)


def _subcentroids(k):
    tris = [np.eye(3)]
    for _ in range(k):
        nt = []
        for t in tris:
            ab, bc, ca = (t[0] + t[1]) / 2, (t[1] + t[2]) / 2, (t[2] + t[0]) / 2
            nt += [np.array([t[0], ab, ca]), np.array([ab, t[1], bc]), np.array([ca, bc, t[2]]), np.array([ab, bc, ca])]
        tris = nt
    return np.array([t.mean(0) for t in tris])


@pytest.fixture(scope="module")
def sphere2():
    V, T = inputs.icosphere(2, 50.0)
    c, a, n = dense.geometry(V, T)
    return V, T, c, a, n


def _pairs_by_class(T, i):
    out = {0: [], 1: [], 2: []}
    for j in range(T.shape[0]):
        if j == i:
            continue
        s = len(set(T[i]) & set(T[j]))
        out[s].append(j)
    return out


def test_double_layer_matches_solid_angle(sphere2):
    # kappa = 0, eps = 2: I2 = int int dG0/dnu_y; the inner integral is -Omega/(4 pi) exactly.
    V, T, c, a, n = sphere2
    ph = dense.Phys(1.0, 2.0, 0.0, qs=4)
    B = _subcentroids(5)
    i = 7
    X = B @ V[T[i]]
    cls = _pairs_by_class(T, i)
    for s, tol in ((1, 2e-3), (2, 2e-3)):
        for j in cls[s][:3]:
            got = dense.pair_integrals(V, T, i, j, ph)[1]
            ref = a[i] * np.mean(-_solid_angle(X, V[T[j]])) / (4 * np.pi)
            assert abs(got - ref) < tol * abs(ref), (s, j, got, ref)
    # identical flat triangle: (x - y) . n = 0, so the K2 and K3 integrals vanish exactly
    I = dense.pair_integrals(V, T, i, i, dense.Phys(1.0, 80.0, 0.1257, qs=3))
    assert I[1] == 0.0 and I[2] == 0.0


def test_double_layer_row_sums_near_minus_half(sphere2):
    # Gauss: for x on a closed surface int dG0/dnu_y dS_y = -1/2; rows of I2 sum to -A_i/2
    # up to the one-point rule's error on regular pairs.
    V, T, c, a, n = sphere2
    ph = dense.Phys(1.0, 2.0, 0.0, qs=4)
    A = dense.assemble(V, T, ph)
    N = T.shape[0]
    I2 = -(A[:N, :N] - np.diag(0.5 * 3.0 * a))
    rs = I2.sum(axis=1) / a
    assert np.all(np.abs(rs + 0.5) < 5e-3)
    # the adjoint double layer has the same row sums (kappa = 0: K3 = (1 - 1/eps) dG0/dnu_x)
    I3 = -(A[N:, N:] - np.diag(0.5 * 1.5 * a)) / 0.5
    assert np.all(np.abs(I3.sum(axis=1) / a + 0.5) < 2e-2)


def test_single_layer_difference_and_k4_match_brute_force(sphere2):
    # K1 = G0 - Gk is bounded and K4 is O(1/r): refined midpoint products converge to the
    # Galerkin integrals of touching pairs.
    V, T, c, a, n = sphere2
    ph = dense.Phys(1.0, 80.0, 0.5, qs=5)
    i = 3
    cls = _pairs_by_class(T, i)
    B = _subcentroids(4)
    for s in (1, 2):
        j = cls[s][0]
        X = B @ V[T[i]]
        Y = B @ V[T[j]]
        K = np.zeros(4)
        for x in X:
            for y in Y:
                K += dense.kernel_point(x, n[i], y, n[j], ph.eps, ph.kappa)
        K *= a[i] * a[j] / (len(X) * len(Y))
        got = dense.pair_integrals(V, T, i, j, ph)
        assert abs(got[0] - K[0]) < 2e-3 * abs(K[0])
        assert abs(got[3] - K[3]) < 3e-2 * abs(K[3]) + 1e-6 * abs(got[1])


def test_kernel_symmetries(sphere2):
    V, T, c, a, n = sphere2
    ph = dense.Phys(1.0, 80.0, 0.1257, qs=3)
    for i, j in ((0, 1), (5, 17), (2, 200)):
        Iij = dense.pair_integrals(V, T, i, j, ph)
        Iji = dense.pair_integrals(V, T, j, i, ph)
        assert abs(Iij[0] - Iji[0]) < 1e-12 * abs(Iij[0])
        assert abs(Iij[3] - Iji[3]) < 1e-12 * abs(Iij[3])
    # kappa = 0: K3 of (i, j) is the transpose of the double layer of (j, i)
    ph0 = dense.Phys(1.0, 4.0, 0.0, qs=3)
    for i, j in ((0, 1), (5, 17), (2, 200)):
        Iij = dense.pair_integrals(V, T, i, j, ph0)
        Iji = dense.pair_integrals(V, T, j, i, ph0)
        assert abs(Iij[2] / (1 - 1 / 4.0) - Iji[1] / (4.0 - 1)) < 1e-12 * abs(Iji[1])


def test_null_case_gives_mass_matrix():
    V, T = inputs.icosphere(1, 3.0)
    ph = dense.Phys(2.0, 2.0, 0.0, qs=3)
    A = dense.assemble(V, T, ph)
    _, a, _ = dense.geometry(V, T)
    assert np.allclose(A, np.diag(np.r_[a, a]), atol=1e-15, rtol=0)


def test_rows_matvec_equals_dense():
    V, T = inputs.icosphere(2, 2.0)
    ph = dense.Phys(1.0, 80.0, 0.1257, qs=3)
    A = dense.assemble(V, T, ph)
    x = inputs.random_density(T.shape[0], 3)
    y = A @ x
    rows = np.array([0, 5, 100, 319])
    y1, y2 = dense.rows_matvec(V, T, ph, rows, x)
    N = T.shape[0]
    assert np.allclose(y1, y[rows], rtol=1e-13, atol=1e-15)
    assert np.allclose(y2, y[N + rows], rtol=1e-13, atol=1e-15)


def test_rhs_gauss_law():
    # int S2 = -Q/eps1 for a closed surface around the charges (centroid rule: O(h^2))
    m = inputs.kirkwood_ball(3, 20.0, 10, 12.0, seed=5)
    ph = dense.Phys(1.0, 80.0, 0.1257)
    b = dense.rhs(m, ph)
    assert abs(b[m.nt:].sum() + m.q.sum()) < 0.02 * np.abs(m.q).sum()
