"""The Cartesian FMM matrix-vector product of Section 2.4, step by step, in plain numpy.

TEST INFRASTRUCTURE. This is the oracle for the CUDA FMM path. It follows the paper's
six-step algorithm (near field, moments, upward pass, interaction phase, downward pass,
evaluation) with the paper's notation, read as follows where the paper leaves a choice:

  * Tree (Section 2.4, cluster hierarchy): the level-0 cube is the smallest axis-parallel
    cube centred on the bounding box of the vertex array. A triangle belongs to the cube of
    each level that holds its centroid (u + v + w)/3. Cells come from
    floor((c - origin) * (1024 / side)), clamped to [0, 1023], interleaved into a 30-bit
    Morton key (x bit above y bit above z bit); elements are ordered by (key, index). All
    leaves sit on one level L: the deepest level whose mean non-empty cluster size is at
    least the leaf size s (or L given explicitly).
  * Shrink scheme: B_c is the bounding box of all vertices of the cluster's triangles, x_c
    its centre, rho_c half its diagonal. Clusters are neighbours when
    (rho_c + rho_c')^2 > eta0^2 |x_c - x_c'|^2, i.e. eta(c, c') > eta0 (def:eta).
  * Lists: N(root) = {root}; at level l the candidates of c are the children of the
    neighbours of its parent; each goes to N(c) or, if not a neighbour, to I(c).
  * Orders p_l = p_L + L - l (variable:order) or p_L at every level.
  * Moments with the one-point rule: m^b(psi_i) = A_i (c_i - x_c)^b and the normal-derivative
    moment A_i n_i . grad (y - x_c)^b at y = c_i (eqmoment, eqmomentL). The four kernels are
    regrouped into two far-field expansions, one of G0 with density
    phi_nu m - phi m_nu and one of Gk with density -phi_nu m + eps phi m_nu (K1 + K2 and
    K3 + K4 of Eq_K1/Eq_K2 share them).
  * MtM (eqMtM); MtL (eqcoeff, with (-1)^|b| and |a| + |b| <= p_l); LtL with the binomial
    shift lambda^b_c' = sum_{a >= b} C(a, b) (x_c' - x_c)^(a-b) lambda^a_c; LtP (LtP) with
    the target-side normal derivative for the dphi/dn rows.
  * Near field: the dense Galerkin entries of ``oracle.dense`` for the element pairs of
    leaf neighbours.

Pins (tests/test_oracle_taylor_fmm.py): with eta0 small enough that every leaf pair is near, the
result equals the dense matvec to rounding; with uniform order the MtM of a cluster equals
its moments computed directly and the LtL equals the re-expanded polynomial; the far-field
error against the dense matvec falls geometrically with p; at p = 8 it is below 1e-4.
"""
from __future__ import annotations

from math import comb, factorial

import numpy as np

from . import dense, taylor

LMAX = 10  # Morton resolution: 2^10 cells per axis


def centroids(verts, tris):
    V = np.asarray(verts, dtype=np.float64)
    T = np.asarray(tris)
    return (V[T[:, 0]] + V[T[:, 1]] + V[T[:, 2]]) / 3.0


def morton_keys(cent, verts):
    """30-bit Morton keys of the centroids in the level-0 cube; returns keys and the cube."""
    V = np.asarray(verts, dtype=np.float64)
    lo = V.min(axis=0)
    hi = V.max(axis=0)
    side = float(np.max(hi - lo))
    ctr = 0.5 * (lo + hi)
    origin = ctr - 0.5 * side
    scale = float(1 << LMAX) / side
    cell = np.floor((cent - origin) * scale)
    cell = np.clip(cell, 0, (1 << LMAX) - 1).astype(np.int64)
    key = np.zeros(cent.shape[0], dtype=np.int64)
    for b in range(LMAX):
        key |= ((cell[:, 0] >> b) & 1) << (3 * b + 2)
        key |= ((cell[:, 1] >> b) & 1) << (3 * b + 1)
        key |= ((cell[:, 2] >> b) & 1) << (3 * b)
    return key, origin, side


class Tree:
    def __init__(self, verts, tris, leaf_size=64, levels=0, eta0=0.8):
        V = np.asarray(verts, dtype=np.float64)
        T = np.asarray(tris, dtype=np.int64)
        N = T.shape[0]
        self.N = N
        cent = centroids(V, T)
        key, self.origin, self.side = morton_keys(cent, V)
        self.order = np.lexsort((np.arange(N), key))  # sorted position -> element index
        ks = key[self.order]
        self.keys = ks

        def bounds(l):
            pre = ks >> (3 * (LMAX - l))
            starts = np.flatnonzero(np.r_[True, pre[1:] != pre[:-1]])
            return starts

        if levels and levels > 0:
            L = int(levels)
        else:
            L = 0
            for l in range(LMAX + 1):
                if N / len(bounds(l)) >= leaf_size:
                    L = l
        self.L = L
        self.begin, self.end = [], []
        for l in range(L + 1):
            st = bounds(l)
            self.begin.append(st)
            self.end.append(np.r_[st[1:], N])
        # parent and children links
        self.parent = [np.zeros(1, dtype=np.int64)]
        self.child_begin, self.child_end = [], []
        for l in range(1, L + 1):
            par = np.searchsorted(self.begin[l - 1], self.begin[l], side="right") - 1
            self.parent.append(par)
        for l in range(L):
            nxt = self.parent[l + 1]
            cb = np.searchsorted(nxt, np.arange(len(self.begin[l])), side="left")
            ce = np.searchsorted(nxt, np.arange(len(self.begin[l])), side="right")
            self.child_begin.append(cb)
            self.child_end.append(ce)
        # shrink boxes
        P = V[T[self.order]]  # (N, 3, 3) sorted
        pmin = P.min(axis=1)
        pmax = P.max(axis=1)
        self.lo = [None] * (L + 1)
        self.hi = [None] * (L + 1)
        self.lo[L] = np.minimum.reduceat(pmin, self.begin[L], axis=0)
        self.hi[L] = np.maximum.reduceat(pmax, self.begin[L], axis=0)
        for l in range(L - 1, -1, -1):
            self.lo[l] = np.minimum.reduceat(self.lo[l + 1], self.child_begin[l], axis=0)
            self.hi[l] = np.maximum.reduceat(self.hi[l + 1], self.child_begin[l], axis=0)
        self.xc = [0.5 * (self.lo[l] + self.hi[l]) for l in range(L + 1)]
        self.rho = []
        for l in range(L + 1):
            d = self.hi[l] - self.lo[l]
            self.rho.append(0.5 * np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]))
        # neighbour and interaction lists
        e2 = eta0 * eta0
        self.near = [[np.array([0], dtype=np.int64)]]
        self.inter = [[np.array([], dtype=np.int64)]]
        for l in range(1, L + 1):
            nl, il = [], []
            for c in range(len(self.begin[l])):
                P_ = self.parent[l][c]
                cand = np.concatenate(
                    [np.arange(self.child_begin[l - 1][q], self.child_end[l - 1][q]) for q in self.near[l - 1][P_]]
                )
                s = self.rho[l][c] + self.rho[l][cand]
                d = self.xc[l][c] - self.xc[l][cand]
                dd = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
                isnear = s * s > e2 * dd
                nl.append(cand[isnear])
                il.append(cand[~isnear])
            self.near.append(nl)
            self.inter.append(il)

    def nclusters(self, l):
        return len(self.begin[l])


def _shift_matrix(idx_hi, idx_lo, t):
    """S[a, b] = C(a, b) t^(a - b) for b <= a (componentwise), a in idx_hi, b in idx_lo."""
    S = np.zeros((len(idx_hi), len(idx_lo)))
    for ia, a in enumerate(idx_hi):
        for ib, b in enumerate(idx_lo):
            if b[0] <= a[0] and b[1] <= a[1] and b[2] <= a[2]:
                S[ia, ib] = (
                    comb(a[0], b[0]) * comb(a[1], b[1]) * comb(a[2], b[2])
                    * t[0] ** (a[0] - b[0]) * t[1] ** (a[1] - b[1]) * t[2] ** (a[2] - b[2])
                )
    return S


def _mono(dvec, idx):
    return np.array([dvec[..., 0] ** a * dvec[..., 1] ** b * dvec[..., 2] ** c for a, b, c in idx]).T


def _dmono(dvec, nrm, idx):
    out = []
    for a, b, c in idx:
        t = np.zeros(dvec.shape[0])
        if a:
            t += nrm[:, 0] * a * dvec[:, 0] ** (a - 1) * dvec[:, 1] ** b * dvec[:, 2] ** c
        if b:
            t += nrm[:, 1] * b * dvec[:, 0] ** a * dvec[:, 1] ** (b - 1) * dvec[:, 2] ** c
        if c:
            t += nrm[:, 2] * c * dvec[:, 0] ** a * dvec[:, 1] ** b * dvec[:, 2] ** (c - 1)
        out.append(t)
    return np.array(out).T


def orders(tree, p, adaptive):
    return [p + (tree.L - l) if adaptive else p for l in range(tree.L + 1)]


def points(tree, verts, tris, ph):
    """The regular rule's points in tree order, element-major (the q^2 points of sorted element
    k at k q^2 ... (k + 1) q^2 - 1): positions, weights 2 A_i w_a, unit normals. Order 1 gives
    the centroids with weights A_i."""
    V = np.asarray(verts, dtype=np.float64)
    T = np.asarray(tris)
    cent, area, nrm = dense.geometry(V, T)
    o = tree.order
    if ph.qr == 1:
        return cent[o], area[o], nrm[o]
    e1, e2, w = ph.rule
    P = V[T[o]]  # (N, 3, 3) corners of the sorted elements
    u, v, ww = P[:, 0, :], P[:, 1, :], P[:, 2, :]
    pos = (u[:, None, :] + e1[None, :, None] * (v - u)[:, None, :] + e2[None, :, None] * (ww - v)[:, None, :])
    wt = 2.0 * area[o][:, None] * w[None, :]
    q2 = len(w)
    return pos.reshape(-1, 3), wt.ravel(), np.repeat(nrm[o], q2, axis=0)


def moments(tree, verts, tris, x, ph, pl, lstop=1):
    """Moments of the two far-field expansions (eqmoment, eqmomentL) at every level from L
    up to lstop: leaf moments by the one-point rule, then the upward pass (eqMtM). For each
    cluster, s0 = sum_i [dphi_i m^b(psi_i) - phi_i m_nu^b(psi_i)] (for G0) and
    sk = sum_i [-dphi_i m^b(psi_i) + eps phi_i m_nu^b(psi_i)] (for Gk), with
    m^b(psi_i) = A_i (c_i - x_c)^b and m_nu^b(psi_i) = A_i n_i . grad (y - x_c)^b at y = c_i.
    pl: the order of each level."""
    N = tree.N
    o = tree.order
    c_s, a_s, n_s = points(tree, verts, tris, ph)
    q2 = len(a_s) // N
    phi, dphi = np.repeat(x[:N][o], q2), np.repeat(x[N:][o], q2)
    eps = ph.eps
    L = tree.L
    idx = [taylor.multi_indices(pl[l]) for l in range(L + 1)]
    s0 = [None] * (L + 1)
    sk = [None] * (L + 1)
    nL = tree.nclusters(L)
    s0[L] = np.zeros((nL, len(idx[L])))
    sk[L] = np.zeros((nL, len(idx[L])))
    for c in range(nL):
        b, e = tree.begin[L][c] * q2, tree.end[L][c] * q2
        dv = c_s[b:e] - tree.xc[L][c]
        M = _mono(dv, idx[L]) * a_s[b:e, None]
        Mn = _dmono(dv, n_s[b:e], idx[L]) * a_s[b:e, None]
        s0[L][c] = dphi[b:e] @ M - phi[b:e] @ Mn
        sk[L][c] = -dphi[b:e] @ M + eps * (phi[b:e] @ Mn)
    # upward pass (MtM); child moments above the child's order are absent
    for l in range(L - 1, lstop - 1, -1):
        nc = tree.nclusters(l)
        s0[l] = np.zeros((nc, len(idx[l])))
        sk[l] = np.zeros((nc, len(idx[l])))
        for c in range(nc):
            for ch in range(tree.child_begin[l][c], tree.child_end[l][c]):
                S = _shift_matrix(idx[l], idx[l + 1], tree.xc[l + 1][ch] - tree.xc[l][c])
                s0[l][c] += S @ s0[l + 1][ch]
                sk[l][c] += S @ sk[l + 1][ch]
    return s0, sk


def treecode_energy(tree, mesh, x, ph, p, theta, adaptive=False):
    """Solvation energy (eqsolengdis) in kcal/mol by the Cartesian treecode of Section 2.5.

    V_n = sum_i A_i [K1(x_n, c_i) dphi_i + K2(x_n, c_i) phi_i] (the one-point rule of the
    direct sum; with ph.qr > 1 the regular rule's points) is accumulated per charge by addCluster from the root: a cluster c whose
    radius and distance to the charge satisfy the MAC (eqMAC) r_c / R <= theta contributes
    its Taylor series (eqsolengformTree) sum_b D^b G(x_n - x_c) (-1)^|b| / b! s[b] for both
    expansions (G0 with s0, Gk with sk, the moments of ``moments``); otherwise its children
    are visited, and a leaf is summed directly. r_c is read as the shrink-box half diagonal
    rho_c, which bounds every point of the cluster, and the test is made in FP64 as
    rho_c^2 <= theta^2 |x_n - x_c|^2. E = 1/2 * 4 pi 332.0716 * sum_n q_n V_n."""
    N = tree.N
    L = tree.L
    o = tree.order
    c_s, a_s, n_s = points(tree, mesh.verts, mesh.tris, ph)
    q2 = len(a_s) // N
    phi, dphi = np.repeat(x[:N][o], q2), np.repeat(x[N:][o], q2)
    eps, kap = ph.eps, ph.kappa
    pl = orders(tree, p, adaptive)
    s0, sk = moments(tree, mesh.verts, mesh.tris, x, ph, pl, lstop=0)
    idx = [taylor.multi_indices(pl[l]) for l in range(L + 1)]
    w = [np.array([(-1.0) ** (a + b + c) / (factorial(a) * factorial(b) * factorial(c)) for a, b, c in idx[l]])
         for l in range(L + 1)]
    th2 = theta * theta
    fpi = 4.0 * np.pi

    def direct(xn, b, e):
        d = xn - c_s[b:e]
        r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
        r = np.sqrt(r2)
        ex = np.exp(-kap * r)
        k1 = (1.0 - ex) / (fpi * r)
        # dG/dnu_y = -g'(r) (n_y . d) / r, g0' = -1 / (4 pi r^2), gk' = -(1 + k r) e^(-k r) / (4 pi r^2)
        nd = n_s[b:e, 0] * d[:, 0] + n_s[b:e, 1] * d[:, 1] + n_s[b:e, 2] * d[:, 2]
        dg0 = nd / (fpi * r2 * r)
        dgk = (1.0 + kap * r) * ex * nd / (fpi * r2 * r)
        k2 = eps * dgk - dg0
        return float(np.sum(a_s[b:e] * (k1 * dphi[b:e] + k2 * phi[b:e])))

    E = 0.0
    for n in range(mesh.nc):
        xn = np.asarray(mesh.qpos[n], dtype=np.float64)
        Vn = 0.0
        accepted = [[] for _ in range(L + 1)]  # clusters whose series is used, by level
        stack = [(0, 0)]
        while stack:
            l, c = stack.pop()
            d = xn - tree.xc[l][c]
            R2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2]
            if tree.rho[l][c] * tree.rho[l][c] <= th2 * R2:
                accepted[l].append(c)
            elif l < L:
                for ch in range(tree.child_end[l][c] - 1, tree.child_begin[l][c] - 1, -1):
                    stack.append((l + 1, ch))
            else:
                Vn += direct(xn, tree.begin[L][c] * q2, tree.end[L][c] * q2)
        # the series of the accepted clusters, one derivative evaluation per level
        for l in range(L + 1):
            if accepted[l]:
                cs = np.array(accepted[l])
                d = xn[None, :] - tree.xc[l][cs]
                D0 = taylor.derivatives(d, pl[l], 0.0)
                Dk = taylor.derivatives(d, pl[l], kap)
                Vn += float(np.sum(D0 * w[l] * s0[l][cs]) + np.sum(Dk * w[l] * sk[l][cs]))
        E += mesh.q[n] * Vn
    return 0.5 * E * fpi * 332.0716


def far_field(tree, verts, tris, x, ph, p, adaptive=False):
    """Far-field part (steps 2-6) of y = A x; returns (y1, y2) in element order."""
    N = tree.N
    o = tree.order
    c_s, a_s, n_s = points(tree, verts, tris, ph)
    q2 = len(a_s) // N
    eps, kap = ph.eps, ph.kappa
    L = tree.L
    pl = orders(tree, p, adaptive)
    idx = [taylor.multi_indices(pl[l]) for l in range(L + 1)]
    y1 = np.zeros(N)
    y2 = np.zeros(N)
    if L == 0:
        return y1, y2
    # steps 2 and 3: leaf moments and the upward pass
    s0, sk = moments(tree, verts, tris, x, ph, pl)
    # step 4: interaction phase (MtL), all pairs of a level at once
    lam0 = [None] * (L + 1)
    lamk = [None] * (L + 1)
    for l in range(1, L + 1):
        nc = tree.nclusters(l)
        lam0[l] = np.zeros((nc, len(idx[l])))
        lamk[l] = np.zeros((nc, len(idx[l])))
        tg = np.concatenate([np.full(len(tree.inter[l][c]), c) for c in range(nc)]).astype(np.int64)
        sr = np.concatenate([tree.inter[l][c] for c in range(nc)]).astype(np.int64)
        if tg.size == 0:
            continue
        d = tree.xc[l][tg] - tree.xc[l][sr]
        D0 = taylor.derivatives(d, pl[l], 0.0)
        Dk = taylor.derivatives(d, pl[l], kap)
        pos = {t: i for i, t in enumerate(idx[l])}
        fac = np.array([factorial(a) * factorial(b) * factorial(c) for a, b, c in idx[l]], dtype=np.float64)
        sgn = np.array([(-1.0) ** (a + b + c) for a, b, c in idx[l]])
        for ia, al in enumerate(idx[l]):
            rest = pl[l] - sum(al)
            bl = [i for i, be in enumerate(idx[l]) if sum(be) <= rest]
            gl = [pos[(al[0] + idx[l][i][0], al[1] + idx[l][i][1], al[2] + idx[l][i][2])] for i in bl]
            w = sgn[bl] / (fac[ia] * fac[bl])
            c0 = np.einsum("pk,pk->p", D0[:, gl] * w, s0[l][sr][:, bl])
            ck = np.einsum("pk,pk->p", Dk[:, gl] * w, sk[l][sr][:, bl])
            np.add.at(lam0[l][:, ia], tg, c0)
            np.add.at(lamk[l][:, ia], tg, ck)
    # step 5: downward pass (LtL)
    for l in range(1, L):
        for c in range(tree.nclusters(l)):
            for ch in range(tree.child_begin[l][c], tree.child_end[l][c]):
                S = _shift_matrix(idx[l], idx[l + 1], tree.xc[l + 1][ch] - tree.xc[l][c])
                lam0[l + 1][ch] += S.T @ lam0[l][c]
                lamk[l + 1][ch] += S.T @ lamk[l][c]
    # step 6: evaluation (LtP), integrated over each target element by the regular rule
    for c in range(tree.nclusters(L)):
        b, e = tree.begin[L][c], tree.end[L][c]
        pb_, pe = b * q2, e * q2
        dv = c_s[pb_:pe] - tree.xc[L][c]
        M = _mono(dv, idx[L])
        Mn = _dmono(dv, n_s[pb_:pe], idx[L])
        y1[b:e] -= (a_s[pb_:pe] * (M @ (lam0[L][c] + lamk[L][c]))).reshape(e - b, q2).sum(axis=1)
        y2[b:e] -= (a_s[pb_:pe] * (Mn @ (lam0[L][c] + lamk[L][c] / eps))).reshape(e - b, q2).sum(axis=1)
    out1 = np.zeros(N)
    out2 = np.zeros(N)
    out1[o] = y1
    out2[o] = y2
    return out1, out2


def near_mask(tree):
    """Boolean (N, N) mask in element order of the pairs handled by the near field."""
    N = tree.N
    L = tree.L
    m = np.zeros((N, N), dtype=bool)
    o = tree.order
    for c in range(tree.nclusters(L)):
        ti = o[tree.begin[L][c]:tree.end[L][c]]
        for c2 in tree.near[L][c]:
            sj = o[tree.begin[L][c2]:tree.end[L][c2]]
            m[np.ix_(ti, sj)] = True
    return m


def matvec(tree, verts, tris, x, ph, p, adaptive=False, A=None):
    """Full FMM product y = A_fmm x = (near block of A) x + far field, for small meshes."""
    N = tree.N
    if A is None:
        A = dense.assemble(verts, tris, ph)
    m = near_mask(tree)
    M2 = np.block([[m, m], [m, m]])
    y = (A * M2) @ x
    f1, f2 = far_field(tree, verts, tris, x, ph, p, adaptive)
    y[:N] += f1
    y[N:] += f2
    return y
