"""Pins of the piecewise-linear (continuous hat function) oracle of Section 2.3 against facts
that do not come from the oracle itself: the partition of unity of the linear functions (which
reduces every 3 x 3 pair block to the pinned piecewise-constant integral), a brute-force
product rule on physical barycentric coordinates for regular pairs, the eigenvalue of the
single-layer operators on a sphere for the spherical harmonic z, symmetry, the closed-form
mass matrix in the null case, and the Kirkwood energy of a centred charge. CPU only."""
import numpy as np
import pytest
from scipy.special import spherical_in, spherical_kn

from oracle import dense, kirkwood, linear
from paper_2110_13778_gb300 import inputs


def _touch_classes(T):
    """one (i, j) pair per class: identical, shared edge, shared vertex, none"""
    out = {3: (0, 0)}
    sets = [set(t) for t in T]
    for j in range(1, len(T)):
        s = len(sets[0] & sets[j])
        out.setdefault(s, (0, j))
    return out


@pytest.mark.parametrize("qr", [1, 2, 4])
def test_partition_of_unity_gives_the_constant_integrals(qr):
    V, T = inputs.perturbed_sphere(2, 3.0, 0.15, seed=7)
    ph = dense.Phys(1.0, 80.0, 0.1257, qs=4, qr=qr)
    cls = _touch_classes(T)
    assert set(cls) == {0, 1, 2, 3}
    for s, (i, j) in cls.items():
        for a, b in ((i, j), (j, i)):
            I1 = linear.pair(V, T, a, b, ph)
            I0 = dense.pair_integrals(V, T, a, b, ph)
            assert np.allclose(I1.sum(axis=(1, 2)), I0, rtol=1e-13, atol=1e-16), (s, a, b)


def _bary(P, x):
    """barycentric coordinates of x in triangle P (3 x 3) from sub-triangle areas"""
    n = np.cross(P[1] - P[0], P[2] - P[0])
    A2 = n @ n
    return np.array([np.cross(P[(k + 1) % 3] - x, P[(k + 2) % 3] - x) @ n / A2 for k in range(3)])


def _stroud(P, n):
    """n^2-point conical product rule on triangle P from numpy's Gauss-Legendre nodes"""
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    A = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
    pts, wts = [], []
    for s, ws in zip(g, w):
        for t, wt in zip(g, w):
            # (u, v) = (s, t (1 - s)) covers the unit triangle, Jacobian (1 - s)
            u, v = s, t * (1.0 - s)
            pts.append(P[0] + u * (P[1] - P[0]) + v * (P[2] - P[0]))
            wts.append(2.0 * A * ws * wt * (1.0 - s))
    return np.array(pts), np.array(wts)


def test_regular_pair_against_brute_force_barycentric_rule():
    V, T = inputs.perturbed_sphere(2, 3.0, 0.15, seed=8)
    ph = dense.Phys(1.0, 80.0, 0.1257, qs=3, qr=4)
    _, _, nrm = dense.geometry(V, T)
    cent = V[T].mean(axis=1)
    i = 0
    d = np.linalg.norm(cent - cent[i], axis=1)
    # a neighbour two rings out (the order-4 rule to ~1e-5) and the farthest element (~1e-10)
    for j, tol in ((int(np.argsort(d)[12]), 1e-4), (int(np.argmax(d)), 1e-9)):
        assert not set(T[i]) & set(T[j])
        got = linear.pair(V, T, i, j, ph)
        Pi, Pj = V[T[i]], V[T[j]]
        xs, wx = _stroud(Pi, 10)
        ys, wy = _stroud(Pj, 10)
        ref = np.zeros((4, 3, 3))
        for x, a in zip(xs, wx):
            lx = _bary(Pi, x)
            for y, b in zip(ys, wy):
                K = dense.kernel_point(x, nrm[i], y, nrm[j], ph.eps, ph.kappa)
                ref += a * b * K[:, None, None] * np.outer(lx, _bary(Pj, y))[None]
        assert np.abs(got - ref).max() < tol * np.abs(ref).max(), (j, np.abs(got - ref).max() / np.abs(ref).max())


def test_symmetric_blocks():
    V, T = inputs.perturbed_sphere(1, 3.0, 0.15, seed=9)
    m = inputs.Mesh(V, T, np.zeros((1, 3)), np.ones(1))
    ph = dense.Phys(1.0, 80.0, 0.1257, qs=4, qr=2)
    A = linear.assemble(m, ph)
    nv = V.shape[0]
    I1, I4 = A[:nv, nv:], A[nv:, :nv]
    assert np.abs(I1 - I1.T).max() < 1e-13 * np.abs(I1).max()
    assert np.abs(I4 - I4.T).max() < 1e-13 * np.abs(I4).max()
    # the product is the assembled matrix applied
    x = np.random.default_rng(3).standard_normal(2 * nv)
    assert np.abs(A @ x - linear.matvec(m, ph, x)).max() < 1e-13 * np.abs(A @ x).max()


def test_null_case_is_the_closed_form_mass_matrix():
    # eps = 1, kappa = 0: every kernel vanishes and A = diag(M, M) with M_ab = int psi_a psi_b
    V, T = inputs.perturbed_sphere(1, 3.0, 0.15, seed=10)
    m = inputs.Mesh(V, T, np.zeros((1, 3)), np.ones(1))
    A = linear.assemble(m, dense.Phys(2.0, 2.0, 0.0, qs=3, qr=2))
    nv = V.shape[0]
    M = linear.mass_matrix(V, T)
    assert np.abs(A[:nv, :nv] - M).max() < 1e-14 * np.abs(M).max()
    assert np.abs(A[nv:, nv:] - M).max() < 1e-14 * np.abs(M).max()
    assert np.abs(A[:nv, nv:]).max() < 1e-15 and np.abs(A[nv:, :nv]).max() < 1e-15
    # and M sums to the surface area
    area = dense.geometry(V, T)[1].sum()
    assert abs(M.sum() - area) < 1e-12 * area


def test_single_layer_eigenvalue_on_a_sphere():
    """int_S G(x, y) z(y) dS_y = mu z(x) on a sphere of radius R with mu = R/3 for G0 and
    (2/pi) kappa R^2 i_1(kappa R) k_1(kappa R) for Gk (addition theorem; modified spherical
    Bessel functions as scipy normalises them): the I1 block applied to the vertex values of z
    must match mu1 M z, the error falling by about 4 per refinement (O(h^2))."""
    R, kap = 2.0, 0.5
    mu1 = R / 3 - (2 / np.pi) * kap * R * R * spherical_in(1, kap * R) * spherical_kn(1, kap * R)
    errs = []
    for lev in (1, 2, 3):
        V, T = inputs.icosphere(lev, R)
        m = inputs.Mesh(V, T, np.zeros((1, 3)), np.ones(1))
        A = linear.assemble(m, dense.Phys(1.0, 80.0, kap, qs=4, qr=2))
        nv = V.shape[0]
        Mz = linear.mass_matrix(V, T) @ V[:, 2]
        errs.append(np.linalg.norm(-A[:nv, nv:] @ V[:, 2] - mu1 * Mz) / np.linalg.norm(mu1 * Mz))
    assert errs[2] < 6.5e-3, errs
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_rhs_and_energy_reduce_to_piecewise_constant():
    m = inputs.kirkwood_ball(2, 2.0, 4, 1.2, seed=11)
    for qr in (1, 3):
        ph = dense.Phys(1.0, 80.0, 0.1257, qs=3, qr=qr)
        nv, nt = m.verts.shape[0], m.nt
        b1, b0 = linear.rhs(m, ph), dense.rhs(m, ph)
        assert abs(b1[:nv].sum() - b0[:nt].sum()) < 1e-12 * np.abs(b0[:nt]).sum()
        assert abs(b1[nv:].sum() - b0[nt:].sum()) < 1e-12 * np.abs(b0[nt:]).sum()
        # constant densities are reproduced exactly by the interpolation
        x1 = np.concatenate([np.full(nv, 0.7), np.full(nv, -0.3)])
        x0 = np.concatenate([np.full(nt, 0.7), np.full(nt, -0.3)])
        e1, e0 = linear.energy(m, ph, x1), dense.energy(m, ph, x0)
        assert abs(e1 - e0) < 1e-12 * abs(e0)


def test_kirkwood_centred_charge():
    a, q = 2.0, 1.0
    ref = kirkwood.centered(q, a, 1.0, 80.0, 0.1257)
    V, T = inputs.icosphere(3, a)
    m = inputs.Mesh(V, T, np.zeros((1, 3)), np.array([q]))
    ph = dense.Phys(1.0, 80.0, 0.1257, qs=3, qr=2)
    x, _, _ = linear.solve(m, ph)
    e1 = linear.energy(m, ph, x)
    x0, _, _ = dense.solve(m, ph)
    e0 = dense.energy(m, ph, x0)
    # both within the discretisation error of a 1280-triangle sphere (Table 1's level);
    # the piecewise-linear solution no worse than the piecewise-constant one
    assert abs(e1 - ref) < 0.02 * abs(ref), (e1, ref)
    assert abs(e1 - ref) <= 1.05 * abs(e0 - ref), (e1, e0, ref)
