"""Pins of the power-series derivative tensors and of the oracle FMM. CPU only."""
from math import factorial

import numpy as np
import pytest

from oracle import dense, fmm, taylor
from paper_2110_13778_gb300 import inputs

KAP = 0.1257


def _G(x, kap):
    r = np.linalg.norm(x)
    return np.exp(-kap * r) / (4 * np.pi * r)


@pytest.mark.parametrize("kap", [0.0, KAP, 1.5])
def test_low_orders_match_closed_forms(kap):
    d = np.array([1.3, -0.7, 2.1])
    idx = taylor.multi_indices(4)
    D = taylor.derivatives(d, 4, kap)
    r = np.linalg.norm(d)
    g = np.exp(-kap * r) / (4 * np.pi * r)
    gp = -(1 + kap * r) * np.exp(-kap * r) / (4 * np.pi * r * r)
    gpp = (2 + 2 * kap * r + (kap * r) ** 2) * np.exp(-kap * r) / (4 * np.pi * r ** 3)
    assert abs(D[0] - g) < 1e-15
    for k in range(3):
        e = [0, 0, 0]
        e[k] = 1
        assert abs(D[idx.index(tuple(e))] - gp * d[k] / r) < 1e-15
    # Hessian: (g'' - g'/r) d_i d_j / r^2 + g'/r delta_ij
    for i in range(3):
        for j in range(3):
            e = [0, 0, 0]
            e[i] += 1
            e[j] += 1
            H = (gpp - gp / r) * d[i] * d[j] / r ** 2 + (gp / r) * (i == j)
            assert abs(D[idx.index(tuple(e))] - H) < 1e-14


def test_matches_finite_differences_order3():
    d = np.array([0.9, 1.7, -1.1])
    idx = taylor.multi_indices(3)
    D = taylor.derivatives(d, 3, KAP)
    h = 2e-3
    for gam in [(3, 0, 0), (1, 1, 1), (2, 0, 1), (0, 1, 2)]:
        # tensor central differences
        tot = 0.0
        steps = [np.eye(3)[k] for k in range(3) for _ in range(gam[k])]
        for signs in np.ndindex(*(2,) * len(steps)):
            s = np.array([1 if b == 0 else -1 for b in signs])
            x = d + sum(si * h * st for si, st in zip(s, steps))
            tot += np.prod(s) * _G(x, KAP)
        fd = tot / (2 * h) ** len(steps)
        assert abs(fd - D[idx.index(gam)]) < 2e-4 * abs(D[idx.index(gam)]) + 1e-9, (gam, fd, D[idx.index(gam)])


@pytest.mark.parametrize("kap", [0.0, KAP])
def test_helmholtz_identity_all_orders(kap):
    # Delta G0 = 0 and Delta Gk = kappa^2 Gk away from the origin, coefficient by coefficient:
    # sum_i D^(g + 2 e_i) G = kappa^2 D^g G for every |g| <= p - 2.
    p = 9
    d = np.array([2.0, -1.0, 0.5])
    idx = taylor.multi_indices(p)
    pos = {t: i for i, t in enumerate(idx)}
    D = taylor.derivatives(d, p, kap)
    for g in idx:
        if sum(g) > p - 2:
            continue
        lap = sum(D[pos[(g[0] + 2 * (k == 0), g[1] + 2 * (k == 1), g[2] + 2 * (k == 2))]] for k in range(3))
        assert abs(lap - kap * kap * D[pos[g]]) < 1e-11 * np.abs(D).max()


def test_kappa_zero_equals_coulomb():
    d = np.array([[1.0, 2.0, 3.0], [0.3, -0.2, 0.9]])
    a = taylor.derivatives(d, 6, 0.0)
    b = taylor.derivatives(d, 6, 1e-300)
    assert np.allclose(a, b, rtol=1e-13)


def test_shift_exactness():
    # MtM: moments about c1 shifted to c2 equal moments about c2 (degree-preserving, exact)
    rng = np.random.default_rng(0)
    y = rng.normal(size=(20, 3))
    w = rng.normal(size=20)
    c1, c2 = np.array([0.1, 0.2, -0.3]), np.array([1.0, -0.5, 0.4])
    idx = taylor.multi_indices(5)
    m1 = w @ fmm._mono(y - c1, idx)
    m2 = w @ fmm._mono(y - c2, idx)
    S = fmm._shift_matrix(idx, idx, c1 - c2)
    assert np.allclose(S @ m1, m2, rtol=1e-12, atol=1e-12)
    # LtL: sum_a lam^a (x - c2)^a re-expanded about c1 evaluates identically
    lam = rng.normal(size=len(idx))
    x = rng.normal(size=(7, 3))
    v2 = fmm._mono(x - c2, idx) @ lam
    S2 = fmm._shift_matrix(idx, idx, c1 - c2)
    v1 = fmm._mono(x - c1, idx) @ (S2.T @ lam)
    assert np.allclose(v1, v2, rtol=1e-11)


@pytest.fixture(scope="module")
def small_sphere():
    V, T = inputs.icosphere(3, 2.0)
    ph = dense.Phys(1.0, 80.0, KAP, qs=3)
    A = dense.assemble(V, T, ph)
    x = inputs.random_density(T.shape[0], 1)
    return V, T, ph, A, x


def test_tree_partitions_all_pairs(small_sphere):
    V, T, ph, A, x = small_sphere
    tr = fmm.Tree(V, T, leaf_size=16, eta0=0.8)
    # each (leaf i, leaf j) pair is covered exactly once: near at the leaf level or by one
    # interaction-list pair of its ancestors
    L = tr.L
    nl = tr.nclusters(L)
    cover = np.zeros((nl, nl), dtype=int)
    anc = [np.arange(nl)]
    for l in range(L, 0, -1):
        anc.insert(0, tr.parent[l][anc[0]])
    for c in range(nl):
        for c2 in tr.near[L][c]:
            cover[c, c2] += 1
    for l in range(1, L + 1):
        for a in range(nl):
            for b in range(nl):
                if anc[l][b] in set(tr.inter[l][anc[l][a]]):
                    cover[a, b] += 1
    assert np.all(cover == 1)
    assert sorted(tr.order.tolist()) == list(range(T.shape[0]))


def test_fmm_all_near_equals_dense(small_sphere):
    V, T, ph, A, x = small_sphere
    tr = fmm.Tree(V, T, leaf_size=16, eta0=1e-9)  # eta > eta0 for every pair: all near
    y = fmm.matvec(tr, V, T, x, ph, 2, A=A)
    assert np.allclose(y, A @ x, rtol=1e-13, atol=1e-13 * np.abs(A @ x).max())


def test_fmm_converges_to_dense(small_sphere):
    V, T, ph, A, x = small_sphere
    y = A @ x
    tr = fmm.Tree(V, T, leaf_size=16, eta0=0.8)
    errs = [np.linalg.norm(fmm.matvec(tr, V, T, x, ph, p, A=A) - y) / np.linalg.norm(y) for p in (2, 4, 6)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4
    # adaptive order is at least as accurate as its finest-level order
    ea = np.linalg.norm(fmm.matvec(tr, V, T, x, ph, 2, adaptive=True, A=A) - y) / np.linalg.norm(y)
    assert ea <= errs[0]


def _one_axis_shifts(v, idx, e, up):
    """Three one-axis passes over the degree-<=p layout idx: x, then y, then z. For each
    output multi-index the pass sums e[axis][|k - j|] v[... j on that axis ...] over j <= k
    (up=False) or j >= k (up=True), staying inside the layout."""
    pos = {a: i for i, a in enumerate(idx)}
    p = max(sum(a) for a in idx)
    for axis in range(3):
        out = np.zeros_like(v)
        for i, a in enumerate(idx):
            s = 0.0
            rng = range(a[axis], p - sum(a) + a[axis] + 1) if up else range(0, a[axis] + 1)
            for j in rng:
                b = list(a)
                b[axis] = j
                s += e[axis][abs(a[axis] - j)] * v[pos[tuple(b)]]
            out[i] = s
        v = out
    return v


def test_scaled_forms_make_translations_one_axis_shifts():
    # the reading behind the GPU translations: with moments stored as (-1)^|b| m / b! (the form
    # the MtL sum consumes), MtM is a shift by e[g] = (-t)^g / g!, one factor per axis; with
    # local coefficients scaled by a!, LtL is the upward shift by t^g / g!
    rng = np.random.default_rng(4)
    p = 6
    idx = taylor.multi_indices(p)
    sgn = np.array([(-1.0) ** sum(a) for a in idx])
    fac = np.array([factorial(a[0]) * factorial(a[1]) * factorial(a[2]) for a in idx], float)
    t = np.array([0.3, -0.7, 0.45])  # x_child - x_parent
    m_child = rng.normal(size=len(idx))
    m_parent = fmm._shift_matrix(idx, idx, t) @ m_child  # eqMtM
    e_m = [[(-t[d]) ** k / factorial(k) for k in range(p + 1)] for d in range(3)]
    got = _one_axis_shifts(sgn * m_child / fac, idx, e_m, up=False)
    assert np.allclose(got, sgn * m_parent / fac, rtol=1e-12, atol=1e-13)
    # LtL: lam_child = S^T lam_parent with S the shift of the child centre relative to the parent
    lam_parent = rng.normal(size=len(idx))
    lam_child = fmm._shift_matrix(idx, idx, t).T @ lam_parent
    e_l = [[t[d] ** k / factorial(k) for k in range(p + 1)] for d in range(3)]
    got = _one_axis_shifts(fac * lam_parent, idx, e_l, up=True)
    assert np.allclose(got, fac * lam_child, rtol=1e-12, atol=1e-12)


def test_scaled_forms_of_leaf_moments_and_evaluation():
    # P2M in the stored form: with e_j[b] = d'^b / b!, d' = x_c - y_j, the moments
    # (-1)^|b| / b! (sum_j w0_j (y_j - x_c)^b - w1_j n_j . grad (y - x_c)^b) equal
    # S[b] + sum_i G_i[b - e_i], S = sum_j w0_j e_j, G_i = sum_j w1_j n_j,i e_j; LtP: the local
    # expansion and its normal derivative from a!-scaled coefficients and e[b] = d^b / b!
    rng = np.random.default_rng(5)
    p = 5
    idx = taylor.multi_indices(p)
    pos = {a: i for i, a in enumerate(idx)}
    fac = np.array([factorial(a[0]) * factorial(a[1]) * factorial(a[2]) for a in idx], float)
    sgn = np.array([(-1.0) ** sum(a) for a in idx])
    xc = np.array([0.2, -0.1, 0.3])
    y = xc + 0.4 * rng.normal(size=(15, 3))
    nrm = rng.normal(size=(15, 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    w0, w1 = rng.normal(size=15), rng.normal(size=15)
    ref = w0 @ fmm._mono(y - xc, idx) - w1 @ fmm._dmono(y - xc, nrm, idx)
    e = fmm._mono(xc - y, idx) / fac  # e_j[b]
    S = w0 @ e
    G = [(w1 * nrm[:, i]) @ e for i in range(3)]
    got = np.array([S[k] + sum(G[i][pos[tuple(a[q] - (q == i) for q in range(3))]]
                               for i in range(3) if a[i] > 0) for k, a in enumerate(idx)])
    assert np.allclose(got, sgn * ref / fac, rtol=1e-12, atol=1e-12)
    # LtP: value and normal derivative of sum_a lam_a (x - x_c)^a at a target with normal n
    lam = rng.normal(size=len(idx))
    x = xc + 0.3 * rng.normal(size=(1, 3))
    n = np.array([[0.6, -0.48, 0.64]])
    val = fmm._mono(x - xc, idx) @ lam
    der = fmm._dmono(x - xc, n, idx) @ lam
    lh = fac * lam
    ex = (fmm._mono(x - xc, idx) / fac)[0]
    up = [[pos.get(tuple(a[q] + (q == i) for q in range(3))) for a in idx] for i in range(3)]
    got_v = np.dot(lh, ex)
    got_d = sum(ex[k] * sum(n[0, i] * lh[up[i][k]] for i in range(3) if up[i][k] is not None)
                for k in range(len(idx)))
    assert np.isclose(got_v, val[0], rtol=1e-12) and np.isclose(got_d, der[0], rtol=1e-11)


def test_treecode_energy_pinned_by_the_direct_sum():
    # Section 2.5's treecode approximates eqsolengdis (the oracle's direct sum): with theta
    # so small that no cluster passes the MAC it is that sum; at theta = 0.5 its error falls
    # geometrically with the order
    m = inputs.kirkwood_ball(3, 20.0, 8, 16.0, seed=6)
    ph = dense.Phys(1.0, 80.0, 0.1257, qs=3)
    x, _, _ = dense.solve(m, ph)
    Ed = dense.energy(m, ph, x)
    tr = fmm.Tree(m.verts, m.tris, leaf_size=16, eta0=0.8)
    assert abs(fmm.treecode_energy(tr, m, x, ph, 4, 1e-9) - Ed) < 1e-13 * abs(Ed)
    errs = [abs(fmm.treecode_energy(tr, m, x, ph, p, 0.5) - Ed) / abs(Ed) for p in (2, 4, 6)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5, errs
    # a wider opening angle accepts more clusters and is less accurate
    assert abs(fmm.treecode_energy(tr, m, x, ph, 4, 0.8) - Ed) / abs(Ed) > errs[1]
