"""Pins of the oracle's singular (touching-pair) Galerkin integrals to 1e-8 and below.

The oracle integrates touching pairs by the Sauter-Schwab transformation to the 4-cube
(Section 2.3, the paragraph after the right-hand side). Here each kernel term it integrates
is computed a second, independent way, and the two must agree far below the discretisation
error, so that a wrong sub-map, Jacobian weight or vertex layout cannot hide:

* G0 = 1/(4 pi r), every class (identical, shared edge, shared vertex): the inner integral
  over the source triangle is the closed-form potential of a uniformly charged flat triangle
  (Wilton, Rao, Glisson, Schaubert, Al-Bundak and Butler, IEEE Trans. Antennas Propag. 32,
  1984), the outer one a tensor Gauss rule on a graded collapsed map of the target triangle.
* Any radial kernel f(r) with F(s) = int_0^s f(t) t dt in closed form: the inner integral in
  polar coordinates about the projection of x onto the source plane, edge by edge, the
  radius done by F and the angle by Gauss-Legendre in psi = asinh(l / h) (smooth in psi).
  Used for K1 = G0 - Gk (all classes) and for K4 of identical (coplanar) pairs, where the
  mixed normal derivative reduces to -g'(r)/r and is radial too.
* dG0/dn on touching pairs: the inner integral is the solid angle of a flat triangle
  (Van Oosterom and Strackee, IEEE Trans. Biomed. Eng. 30, 1983).

The outer rule: x = A + u (B - A) + u v (C - B) with u and v graded by the quintic
smoothstep (first and second derivatives vanish at both ends), which turns the r log r and
log behaviour of the inner integrals at the edges and corners into a smooth integrand.
CPU only.
"""
import numpy as np
import pytest

from oracle import dense
from paper_2110_13778_gb300 import inputs

KAPPA = 0.1257


def _gl01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _outer_rule(P, n=60):
    """Points and weights of a rule for int_tau g(x) dS_x, tau = triangle P (3 x 3)."""
    A, B, C = P
    a, wa = _gl01(n)
    s = a ** 3 * (10.0 - 15.0 * a + 6.0 * a * a)
    ds = 30.0 * a * a * (1.0 - a) ** 2
    U, Vv = np.meshgrid(s, s, indexing="ij")
    W = np.outer(wa * ds, wa * ds)
    X = A + U[..., None] * (B - A) + (U * Vv)[..., None] * (C - B)
    area = 0.5 * np.linalg.norm(np.cross(B - A, C - A))
    return X.reshape(-1, 3), (W * U * 2.0 * area).ravel()


def _edges(P):
    A, B, C = P
    n = np.cross(B - A, C - A)
    n /= np.linalg.norm(n)
    return n, ((A, B), (B, C), (C, A))


def _wilton_potential(X, P):
    """int_tau 1/|x - y| dS_y for each row x of X (uniformly charged flat triangle)."""
    n, edges = _edges(P)
    w0 = (X - P[0]) @ n
    rho = X - w0[:, None] * n
    aw = np.abs(w0)
    tot = np.zeros(len(X))
    for a, b in edges:
        lhat = (b - a) / np.linalg.norm(b - a)
        uhat = np.cross(lhat, n)  # in-plane outward normal of the edge
        lp, lm = (b - rho) @ lhat, (a - rho) @ lhat
        d = (a - rho) @ uhat
        P0 = np.abs(d)
        R02 = P0 ** 2 + w0 ** 2
        R0 = np.sqrt(R02)
        ok = R0 > 0
        R0s = np.where(ok, R0, 1.0)
        Rp, Rm = np.linalg.norm(X - b, axis=1), np.linalg.norm(X - a, axis=1)
        # ln((R+ + l+)/(R- + l-)) written as a difference of asinh (no cancellation)
        t1 = np.where(ok, P0 * (np.arcsinh(lp / R0s) - np.arcsinh(lm / R0s)), 0.0)
        t2 = aw * (np.arctan2(P0 * lp, R02 + aw * Rp) - np.arctan2(P0 * lm, R02 + aw * Rm))
        tot += np.sign(d) * (t1 - t2)
    return tot


def _polar_radial(X, P, F, npsi=64):
    """int_tau f(|x - y|) dS_y for each row x of X, given F(s) = int_0^s f(t) t dt."""
    n, edges = _edges(P)
    w0 = (X - P[0]) @ n
    rho = X - w0[:, None] * n
    g, gw = _gl01(npsi)
    tot = np.zeros(len(X))
    Fw = F(np.abs(w0))
    for a, b in edges:
        lhat = (b - a) / np.linalg.norm(b - a)
        uhat = np.cross(lhat, n)
        lp, lm = (b - rho) @ lhat, (a - rho) @ lhat
        d = (a - rho) @ uhat
        h = np.abs(d)
        ok = h > 0
        hs = np.where(ok, h, 1.0)
        pp, pm = np.arcsinh(lp / hs), np.arcsinh(lm / hs)
        psi = pm[:, None] + (pp - pm)[:, None] * g[None, :]
        ch = np.cosh(psi)
        s = np.sqrt((hs[:, None] * ch) ** 2 + w0[:, None] ** 2)
        val = (F(s) - Fw[:, None]) / ch
        tot += np.where(ok, np.sign(d) * (val @ gw) * (pp - pm), 0.0)
    return tot


def _solid_angle(X, P):
    """Signed solid angle of triangle P seen from the rows of X (Van Oosterom-Strackee)."""
    R = P[None, :, :] - X[:, None, :]
    r = np.linalg.norm(R, axis=2)
    num = np.einsum("ij,ij->i", R[:, 0], np.cross(R[:, 1], R[:, 2]))
    den = (r[:, 0] * r[:, 1] * r[:, 2] + np.einsum("ij,ij->i", R[:, 0], R[:, 1]) * r[:, 2]
           + np.einsum("ij,ij->i", R[:, 0], R[:, 2]) * r[:, 1] + np.einsum("ij,ij->i", R[:, 1], R[:, 2]) * r[:, 0])
    return 2.0 * np.arctan2(num, den)


def _series(t, coef):
    out = np.zeros_like(t)
    for c in coef[::-1]:
        out = out * t + c
    return out


# F(s) = int_0^s f(t) t dt for the radial kernels, with Taylor forms where kappa s is small
def _F_g0(s):
    return s / (4.0 * np.pi)


def _F_k1(s, k=KAPPA):
    # f = (1 - exp(-k r)) / (4 pi r):  F = (s - (1 - exp(-k s)) / k) / (4 pi)
    t = k * s
    big = (s + np.expm1(-t) / k) / (4.0 * np.pi)
    small = t * t * _series(t, [1 / 2, -1 / 6, 1 / 24, -1 / 120, 1 / 720, -1 / 5040]) / k / (4.0 * np.pi)
    return np.where(t < 1e-2, small, big)


def _F_k4_coplanar(s, k=KAPPA):
    # coplanar pair: K4 = -(gk' - g0')/r = -(1 - (1 + k r) exp(-k r)) / (4 pi r^3);
    # F = -(k + (exp(-k s) - 1) / s) / (4 pi)
    t = k * s
    with np.errstate(divide="ignore", invalid="ignore"):
        big = -(k + np.expm1(-t) / s) / (4.0 * np.pi)
    small = -k * t * _series(t, [1 / 2, -1 / 6, 1 / 24, -1 / 120, 1 / 720, -1 / 5040]) / (4.0 * np.pi)
    return np.where(t < 1e-2, small, big)


@pytest.fixture(scope="module")
def mesh():
    # an irregular closed surface: icosphere vertices moved at random (no two touching
    # triangles coplanar, edge ratios up to ~2)
    V, T = inputs.icosphere(2, 50.0)
    V = V + np.random.default_rng(1).normal(scale=0.8, size=V.shape)
    return V, T


def _touching(T, i):
    out = {1: [], 2: [], 3: [i]}
    for j in range(T.shape[0]):
        if j != i:
            s = len(set(T[i]) & set(T[j]))
            if s:
                out[s].append(j)
    return out


def _pairs(T):
    pairs = []
    for i in (7, 101):
        cls = _touching(T, i)
        pairs += [(3, i, i)] + [(2, i, j) for j in cls[2][:2]] + [(1, i, j) for j in cls[1][:3]]
    return pairs


def test_reference_methods_agree(mesh):
    # the polar method with F = s / (4 pi) and the closed-form potential are two routes to
    # the same inner integral; both against a plain midpoint sum far from the triangle
    V, T = mesh
    P = V[T[7]]
    X, _ = _outer_rule(V[T[8]], 12)
    X = np.vstack([X, P.mean(0) + np.array([[0.3, 0.2, 0.1], [5.0, -3.0, 2.0]])])
    assert np.allclose(_wilton_potential(X, P) / (4 * np.pi), _polar_radial(X, P, _F_g0), rtol=1e-12, atol=1e-14)
    far = P.mean(0) + np.array([[400.0, 300.0, -200.0]])
    Y, W = _outer_rule(P, 30)
    brute = W @ (1.0 / np.linalg.norm(Y - far, axis=1))
    assert abs(_wilton_potential(far, P)[0] - brute) < 1e-12 * brute


def test_g0_single_layer_all_classes(mesh):
    V, T = mesh
    for cls, i, j in _pairs(T):
        a, b = min(i, j), max(i, j)
        X, W = _outer_rule(V[T[a]])
        ref = W @ _wilton_potential(X, V[T[b]]) / (4 * np.pi)
        errs = []
        for qs in (4, 6, 8, 12):
            got = dense.pair_terms(V, T, i, j, KAPPA, qs)[6]
            errs.append(abs(got - ref) / abs(ref))
        # exponential convergence in the Gauss order: 1e-7 at qs = 6, 1e-8 at 8, 1e-11 at 12
        assert errs[1] < 1e-7 and errs[2] < 1e-8 and errs[3] < 1e-11, (cls, j, errs)
        assert errs[3] < errs[2] < errs[0], (cls, j, errs)


def test_k1_all_classes(mesh):
    # K1 = G0 - Gk, the single-layer difference of eq_linsysEntry's A12 block
    V, T = mesh
    for cls, i, j in _pairs(T):
        a, b = min(i, j), max(i, j)
        X, W = _outer_rule(V[T[a]])
        ref = W @ _polar_radial(X, V[T[b]], _F_k1)
        got6 = dense.pair_terms(V, T, i, j, KAPPA, 6)[0]
        got8 = dense.pair_terms(V, T, i, j, KAPPA, 8)[0]
        got12 = dense.pair_terms(V, T, i, j, KAPPA, 12)[0]
        assert abs(got6 - ref) < 1e-8 * abs(ref), (cls, j, got6, ref)
        assert abs(got8 - ref) < 1e-9 * abs(ref), (cls, j, got8, ref)
        assert abs(got12 - ref) < 1e-11 * abs(ref), (cls, j, got12, ref)
        # the pair integral the matrix uses is this term
        I = dense.pair_integrals(V, T, i, j, dense.Phys(1.0, 80.0, KAPPA, qs=8))
        assert I[0] == got8


def test_k4_identical_pairs(mesh):
    # identical flat triangle: (x - y).n = 0, n_x . n_y = 1, so K4 = -(gk'(r) - g0'(r))/r
    V, T = mesh
    for i in (7, 101, 250):
        X, W = _outer_rule(V[T[i]])
        ref = W @ _polar_radial(X, V[T[i]], _F_k4_coplanar)
        got = dense.pair_terms(V, T, i, i, KAPPA, 8)[1]
        got12 = dense.pair_terms(V, T, i, i, KAPPA, 12)[1]
        assert abs(got - ref) < 1e-8 * abs(ref), (i, got, ref)
        assert abs(got12 - ref) < 1e-11 * abs(ref), (i, got12, ref)
        I = dense.pair_integrals(V, T, i, i, dense.Phys(1.0, 80.0, KAPPA, qs=8))
        assert I[3] == got


def test_g0_double_layer_touching_pairs(mesh):
    # int_{tau_b} dG0/dn_y dS_y = -Omega_b(x) / (4 pi) and, with the roles exchanged,
    # int_{tau_a} dG0/dn_x dS_x = -Omega_a(y) / (4 pi)
    V, T = mesh
    for cls, i, j in _pairs(T):
        if cls == 3:
            continue
        a, b = min(i, j), max(i, j)
        X, W = _outer_rule(V[T[a]])
        ref_y = W @ (-_solid_angle(X, V[T[b]]) / (4 * np.pi))
        Y, Wy = _outer_rule(V[T[b]])
        ref_x = Wy @ (-_solid_angle(Y, V[T[a]]) / (4 * np.pi))
        for qs, tol in ((8, 1e-8), (12, 1e-11)):
            t = dense.pair_terms(V, T, i, j, KAPPA, qs)
            scale = abs(t[6]) / 50.0  # the double layer of a touching pair can nearly vanish
            assert abs(t[2] - ref_y) < tol * max(abs(ref_y), scale), (cls, j, qs, t[2], ref_y)
            assert abs(t[4] - ref_x) < tol * max(abs(ref_x), scale), (cls, j, qs, t[4], ref_x)


def test_a_planted_weight_error_is_caught(mesh):
    # what the pins guard against: one identical-pair sub-map weighted 1 % high moves the
    # G0 integral by ~0.2 %, five orders above the pin's bound
    V, T = mesh
    X, W = _outer_rule(V[T[7]])
    ref = W @ _wilton_potential(X, V[T[7]]) / (4 * np.pi)
    gx, gw = dense.gauss_legendre01(8)
    P = V[T[7]]
    area = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    tot = 0.0
    for a in range(8):
        for b in range(8):
            for c in range(8):
                for d in range(8):
                    xh, yh, jac = dense.ss_points(3, gx[a], gx[b], gx[c], gx[d])
                    w = gw[a] * gw[b] * gw[c] * gw[d] * jac * np.where(np.arange(len(jac)) == 2, 1.01, 1.0)
                    x = P[0] + xh[:, :1] * (P[1] - P[0]) + xh[:, 1:] * (P[2] - P[1])
                    y = P[0] + yh[:, :1] * (P[1] - P[0]) + yh[:, 1:] * (P[2] - P[1])
                    tot += np.sum(w / np.linalg.norm(x - y, axis=1))
    planted = tot * (2 * area) ** 2 / (4 * np.pi)
    assert abs(planted - ref) > 1e-3 * abs(ref)
