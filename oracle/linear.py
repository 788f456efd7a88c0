"""Piecewise-linear Galerkin system: continuous hat functions S^1_h (Section 2.3, eqlinearfcn
and eqglinearcfcn).

TEST INFRASTRUCTURE (see the package header). The unknowns live at the vertices,
x = [phi_1..phi_nv ; dphi_1..dphi_nv]; entries are the element-pair integrals of the kernels
weighted by the linear functions of both elements (regular pairs by the rule of ``Phys.qr``,
touching pairs by the same Sauter-Schwab quadrature as the piecewise-constant system) summed
onto vertices, and the identity term is the mass matrix int psi_a psi_b. All of it is C
(``pb_oracle.c``, the ``orc_p1_*`` functions).

Pins (tests/test_oracle_linear.py):
  * partition of unity: the three linear functions of an element sum to 1, so summing a
    pair's 3 x 3 integrals gives the piecewise-constant integral of the pinned oracle, for
    regular and for all three touching classes;
  * the single-layer operator of a sphere has the spherical harmonics as eigenfunctions,
    int_S Y_l(y) / (4 pi |x - y|) dS_y = R Y_l(x) / (2 l + 1); with u = z (l = 1) the
    piecewise-linear Galerkin residual against R z / 3 falls by about 4 per refinement
    (O(h^2), where the piecewise-constant one falls by about 2);
  * symmetry: the G0 - Gk and mixed-derivative blocks are symmetric matrices;
  * the mass matrix against its closed form, and the Kirkwood energy of a centred charge:
    the piecewise-linear solve lands within the piecewise-constant error at the same mesh.
"""
from __future__ import annotations

import numpy as np

from . import lib
from .dense import Phys, _dp, _f64, _i32


def pair(verts, tris, i, j, ph: Phys):
    """I[m][a][b], m = K1..K4, a a corner of target i, b a corner of source j (uploaded order)."""
    out = np.zeros(36)
    lib().orc_p1_pair_integrals(_dp(_f64(verts)), _ip32(tris), int(i), int(j), ph.eps, ph.kappa, ph.qs,
                                *ph.rule_args(), _dp(out))
    return out.reshape(4, 3, 3)


def pair_terms(verts, tris, i, j, kappa, qs):
    """The eight Sauter-Schwab term integrals of a touching pair, weighted by the linear
    functions: out[m][a][b] with a a corner of min(i, j) and b a corner of max(i, j)."""
    out = np.zeros(72)
    if lib().orc_p1_pair_terms(_dp(_f64(verts)), _ip32(tris), int(i), int(j), float(kappa), int(qs), _dp(out)) < 0:
        raise ValueError("not a touching pair, or bad quadrature order")
    return out.reshape(8, 3, 3)


def _ip32(tris):
    return tris_ptr(_i32(tris))


def tris_ptr(T):
    import ctypes

    return T.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def nverts(mesh):
    return int(np.asarray(mesh.verts).shape[0])


def matvec(mesh, ph: Phys, x):
    """y = A x of the piecewise-linear system (length 2 nv)."""
    V, T = _f64(mesh.verts), _i32(mesh.tris)
    nv = V.shape[0]
    y = np.zeros(2 * nv)
    lib().orc_p1_matvec(_dp(V), tris_ptr(T), T.shape[0], nv, ph.eps, ph.kappa, ph.qs, *ph.rule_args(),
                        _dp(_f64(x)), _dp(y))
    return y


def assemble(mesh, ph: Phys):
    """Dense 2 nv x 2 nv matrix (small meshes)."""
    V, T = _f64(mesh.verts), _i32(mesh.tris)
    nv = V.shape[0]
    A = np.zeros((2 * nv, 2 * nv))
    lib().orc_p1_assemble(_dp(V), tris_ptr(T), T.shape[0], nv, ph.eps, ph.kappa, ph.qs, *ph.rule_args(), _dp(A))
    return A


def rhs(mesh, ph: Phys):
    V, T = _f64(mesh.verts), _i32(mesh.tris)
    nv = V.shape[0]
    b = np.zeros(2 * nv)
    lib().orc_p1_rhs(_dp(V), tris_ptr(T), T.shape[0], nv, _dp(_f64(mesh.qpos)), _dp(_f64(mesh.q)), mesh.nc,
                     ph.eps1, *ph.rule_args(), _dp(b))
    return b


def energy(mesh, ph: Phys, x):
    """Solvation energy (eqsolengdis) in kcal/mol of a piecewise-linear solution."""
    V, T = _f64(mesh.verts), _i32(mesh.tris)
    return float(lib().orc_p1_energy(_dp(V), tris_ptr(T), T.shape[0], V.shape[0], _dp(_f64(mesh.qpos)),
                                     _dp(_f64(mesh.q)), mesh.nc, ph.eps, ph.kappa, *ph.rule_args(), _dp(_f64(x))))


def mass_matrix(verts, tris):
    """int psi_a psi_b, assembled from the closed form A (1 + [a == b]) / 12 per element."""
    V, T = np.asarray(verts, dtype=np.float64), np.asarray(tris)
    nv = V.shape[0]
    M = np.zeros((nv, nv))
    for t in T:
        A = 0.5 * np.linalg.norm(np.cross(V[t[1]] - V[t[0]], V[t[2]] - V[t[0]]))
        for a in range(3):
            for b in range(3):
                M[t[a], t[b]] += A * (2.0 if a == b else 1.0) / 12.0
    return M


def solve(mesh, ph: Phys, A=None):
    """Dense LU solve of the piecewise-linear system."""
    if A is None:
        A = assemble(mesh, ph)
    b = rhs(mesh, ph)
    return np.linalg.solve(A, b), A, b
