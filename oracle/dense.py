"""Dense Galerkin system of Section 2.3 (def:linsys, eq_linsysEntry), solved by LU.

TEST INFRASTRUCTURE (see the package header). Pins:
  * pair integrals (tests/test_oracle_dense.py) -- Sauter-Schwab sub-maps integrate
    polynomials on tau x tau exactly; coplanar identical pairs give exactly zero K2/K3
    integrals; K1/K4 blocks are symmetric; double layers of adjacent pairs against solid
    angles, K1/K4 against refined midpoint products;
  * singular terms (tests/test_oracle_singular_pins.py) -- the G0 part of identical,
    edge- and vertex-adjacent pairs against the closed-form potential of a uniformly charged
    flat triangle with a graded outer Gauss rule; K1 (all classes) and K4 (identical pairs)
    against polar-coordinate integrals with closed-form radial parts; dG0/dn of adjacent
    pairs against solid angles; 1e-8 at qs = 8 and 1e-11 at qs = 12.
  * solve + energy -- Kirkwood closed form (centred charge) and Kirkwood series (off-centre
    charges) within the discretisation error the paper prints in Table 1; the null case
    eps = 1, kappa = 0 gives A = mass matrix and E = 0.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib

KCAL = 4.0 * np.pi * 332.0716  # e_c/(4 pi A) -> kcal/mol/e_c (Section 3)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _golub_welsch(a, b, mu0):
    """Gauss rule of the orthogonal polynomials with monic recurrence coefficients a_k (k < n)
    and b_k (1 <= k < n), total weight mu0: nodes are the eigenvalues of the symmetric
    tridiagonal Jacobi matrix, weights mu0 times the squared first eigenvector components
    (Golub and Welsch, Math. Comp. 23, 1969)."""
    J = np.diag(np.asarray(a, dtype=np.float64))
    if len(a) > 1:
        off = np.sqrt(np.asarray(b, dtype=np.float64))
        J += np.diag(off, 1) + np.diag(off, -1)
    x, vec = np.linalg.eigh(J)
    return x, mu0 * vec[0, :] ** 2


def triangle_rule(q):
    """Order-q regular rule on the reference triangle {0 <= e2 <= e1 <= 1} (q^2 points, the
    "tensor product Gauss rule" of Section 3.1 read as a collapsed product): Gauss-Jacobi with
    weight e1 in e1 (the Jacobian of e2 = e1 s) times Gauss-Legendre in s = e2 / e1. Exact for
    polynomials of total degree <= 2q - 1; q = 1 is the centroid (2/3, 1/3) with weight 1/2.
    Returns (e1, e2, w), weights summing to 1/2."""
    k = np.arange(q)
    kk = np.arange(1, q)
    # weight t on [0, 1]: the Jacobi (alpha, beta) = (0, 1) recurrence on [-1, 1], shifted
    a_t = (1.0 / ((2 * k + 1) * (2 * k + 3)) + 1.0) / 2.0
    b_t = kk * (kk + 1) / (2.0 * kk + 1) ** 2 / 4.0
    t, wt = _golub_welsch(a_t, b_t, 0.5)
    # weight 1 on [0, 1]: Legendre, shifted
    a_s = np.full(q, 0.5)
    b_s = kk * kk / (4.0 * kk * kk - 1.0) / 4.0
    sv, ws = _golub_welsch(a_s, b_s, 1.0)
    e1 = np.repeat(t, q)
    e2 = e1 * np.tile(sv, q)
    w = np.outer(wt, ws).ravel()
    if q == 1:  # exactly the centroid
        e1, e2, w = np.array([2.0 / 3.0]), np.array([1.0 / 3.0]), np.array([0.5])
    return e1, e2, w


class Phys:
    """eps1 (inside), eps2 (outside), kappa (1/Angstrom), qs (Gauss points per cube axis of
    the singular quadrature), qr (order of the regular rule of non-touching pairs, the
    right-hand side and the energy: 1 = centroid, 2-4 = Table 2's orders)."""

    def __init__(self, eps1=1.0, eps2=80.0, kappa=0.1257, qs=3, qr=1):
        self.eps1, self.eps2, self.kappa, self.qs = float(eps1), float(eps2), float(kappa), int(qs)
        self.qr = int(qr)
        self.rule = triangle_rule(self.qr)

    @property
    def eps(self):
        return self.eps2 / self.eps1

    def rule_args(self):
        e1, e2, w = self.rule
        return (len(w), _dp(e1), _dp(e2), _dp(w))


def gauss_legendre01(n):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().orc_gauss_legendre01(n, _dp(x), _dp(w)) != 0:
        raise ValueError("order out of range")
    return x, w


def kernel_point(x, nx, y, ny, eps, kappa):
    out = np.zeros(4)
    lib().orc_kernel_point(_dp(_f64(x)), _dp(_f64(nx)), _dp(_f64(y)), _dp(_f64(ny)), eps, kappa, _dp(out))
    return out


def geometry(verts, tris):
    V, T = _f64(verts), _i32(tris)
    nt = T.shape[0]
    c = np.zeros((nt, 3))
    a = np.zeros(nt)
    n = np.zeros((nt, 3))
    lib().orc_geometry(_dp(V), _ip(T), nt, _dp(c), _dp(a), _dp(n))
    return c, a, n


def ss_points(case, xi, h1, h2, h3):
    xh = np.zeros(12)
    yh = np.zeros(12)
    jac = np.zeros(6)
    k = lib().orc_ss_points(case, xi, h1, h2, h3, _dp(xh), _dp(yh), _dp(jac))
    return xh[: 2 * k].reshape(k, 2), yh[: 2 * k].reshape(k, 2), jac[:k]


def pair_integrals(verts, tris, i, j, ph: Phys):
    V, T = _f64(verts), _i32(tris)
    out = np.zeros(4)
    lib().orc_pair_integrals(_dp(V), _ip(T), int(i), int(j), ph.eps, ph.kappa, ph.qs, *ph.rule_args(), _dp(out))
    return out


def pair_terms(verts, tris, i, j, kappa, qs):
    """Sauter-Schwab integrals over tau_a x tau_b (a = min(i, j) carries x, b = max(i, j)
    carries y) of the eight kernel terms [G0 - Gk, d2Gk/dnx dny - d2G0/dnx dny, dG0/dny,
    dGk/dny, dG0/dnx, dGk/dnx, G0, Gk] of a touching pair: the numbers the pair integrals are
    made of, exposed so that each can be pinned on its own."""
    V, T = _f64(verts), _i32(tris)
    out = np.zeros(8)
    if lib().orc_pair_terms(_dp(V), _ip(T), int(i), int(j), float(kappa), int(qs), _dp(out)) < 0:
        raise ValueError("not a touching pair, or bad quadrature order")
    return out


def assemble(verts, tris, ph: Phys):
    """Dense 2N x 2N matrix, unknowns ordered [phi; dphi/dn]."""
    V, T = _f64(verts), _i32(tris)
    nt = T.shape[0]
    A = np.zeros((2 * nt, 2 * nt))
    lib().orc_assemble(_dp(V), _ip(T), nt, ph.eps, ph.kappa, ph.qs, *ph.rule_args(), _dp(A))
    return A


def rows_matvec(verts, tris, ph: Phys, elems, x):
    """(A x) restricted to the phi and dphi/dn rows of the given elements: returns (y1, y2)."""
    V, T = _f64(verts), _i32(tris)
    e = _i32(elems)
    xx = _f64(x)
    y = np.zeros(2 * e.shape[0])
    lib().orc_rows_matvec(_dp(V), _ip(T), T.shape[0], ph.eps, ph.kappa, ph.qs, *ph.rule_args(), e.shape[0], _ip(e),
                          _dp(xx), _dp(y))
    return y[0::2].copy(), y[1::2].copy()


def rhs(mesh, ph: Phys):
    V, T = _f64(mesh.verts), _i32(mesh.tris)
    b = np.zeros(2 * T.shape[0])
    lib().orc_rhs(_dp(V), _ip(T), T.shape[0], _dp(_f64(mesh.qpos)), _dp(_f64(mesh.q)), mesh.nc, ph.eps1,
                  *ph.rule_args(), _dp(b))
    return b


def energy(mesh, ph: Phys, x):
    """Solvation energy (eqsolengdis) in kcal/mol."""
    V, T = _f64(mesh.verts), _i32(mesh.tris)
    xx = _f64(x)
    return float(
        lib().orc_energy(_dp(V), _ip(T), T.shape[0], _dp(_f64(mesh.qpos)), _dp(_f64(mesh.q)), mesh.nc, ph.eps, ph.kappa,
                         *ph.rule_args(), _dp(xx))
    )


def matvec(mesh, ph: Phys, x):
    """The full product A x of def:linsys by rows (no matrix stored): [y1; y2]."""
    y1, y2 = rows_matvec(mesh.verts, mesh.tris, ph, np.arange(mesh.nt), x)
    return np.concatenate([y1, y2])


def solve_matrix_free(mesh, ph: Phys, tol=1e-11, restart=60, maxiter=40):
    """A x = b for meshes whose dense matrix does not fit: restarted GMRES (scipy, FP64) over
    the row-by-row product above, right-scaled by the diagonal of mass terms
    D = diag(1/2 (1+eps) A_i, 1/2 (1+1/eps) A_i) (the diagonal preconditioner of Section 2.6
    without its integral part): A D^-1 z = b, x = D^-1 z, so the stopping test is on the true
    residual. Returns (x, b, relative residual ||b - A x|| / ||b|| recomputed with one more
    product, products used)."""
    from scipy.sparse.linalg import LinearOperator, gmres

    n = 2 * mesh.nt
    _, area, _ = geometry(mesh.verts, mesh.tris)
    d = np.concatenate([0.5 * (1.0 + ph.eps) * area, 0.5 * (1.0 + 1.0 / ph.eps) * area])
    count = [0]

    def mv(z):
        count[0] += 1
        return matvec(mesh, ph, np.asarray(z, dtype=np.float64).ravel() / d)

    b = rhs(mesh, ph)
    op = LinearOperator((n, n), matvec=mv, dtype=np.float64)
    z, info = gmres(op, b, rtol=tol, atol=0.0, restart=restart, maxiter=maxiter)
    x = z / d
    res = np.linalg.norm(b - matvec(mesh, ph, x)) / np.linalg.norm(b)
    return x, b, float(res), count[0] + 1


def solve(mesh, ph: Phys, A=None):
    """Dense LU solve of A x = b (partial pivoting, LAPACK via numpy)."""
    if A is None:
        A = assemble(mesh.verts, mesh.tris, ph)
    b = rhs(mesh, ph)
    x = np.linalg.solve(A, b)
    return x, A, b
