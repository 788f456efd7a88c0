"""Parity of the CUDA path (through the C ABI) with the CPU oracle. Needs a GPU.

Tolerances: integer work (tree order, cluster ranges, lists) bit-exact; FP64 mode within
1e-10 relative L2 of the oracle computing the same algorithm; mixed precision within 2e-5
(FP32 arithmetic with FP64 leaf sums); FMM against the dense Galerkin matvec within 1e-4 at
p = 8 (the required accuracy of the method); energies within 1e-3 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, fmm, kirkwood  # noqa: E402
from paper_2110_13778_gb300 import inputs, pb  # noqa: E402

pytestmark = pytest.mark.gpu

KAP = 0.1257


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_13778_gb300 import build

    build.build()
    pb.lib()


def _ctx(mesh, **kw):
    prm = pb.params(**kw)
    ctx = pb.pb_create(prm)
    pb.pb_mesh_upload(ctx, mesh.verts, mesh.tris, mesh.qpos, mesh.q)
    pb.pb_build_tree(ctx)
    return ctx


def _dev(x):
    return torch.tensor(np.asarray(x), device="cuda", dtype=torch.float64)


@pytest.fixture(scope="module")
def sphere3():
    m = inputs.kirkwood_ball(3, 2.0, 5, 1.5, seed=3)
    ph = dense.Phys(1.0, 80.0, KAP, qs=3)
    A = dense.assemble(m.verts, m.tris, ph)
    return m, ph, A


@pytest.mark.parametrize("leaf,eta0", [(16, 0.8), (32, 0.5), (8, 0.7)])
def test_tree_bit_exact(sphere3, leaf, eta0):
    m, ph, A = sphere3
    ctx = _ctx(m, leaf_size=leaf, eta0=eta0)
    try:
        st, order, lb, nc, ni, ic, ii = pb.pb_get_tree(ctx, m.nt)
        tr = fmm.Tree(m.verts, m.tris, leaf_size=leaf, eta0=eta0)
        assert st["levels"] == tr.L
        assert np.array_equal(order, tr.order)
        off = 0
        noff = ioff = 0
        for l in range(tr.L + 1):
            n = tr.nclusters(l)
            assert st["nclusters"][l] == n
            assert np.array_equal(lb[off:off + n], tr.begin[l])
            for c in range(n):
                near = ni[noff:noff + nc[off + c]]
                inter = ii[ioff:ioff + ic[off + c]]
                assert np.array_equal(near, tr.near[l][c]), (l, c)
                assert np.array_equal(inter, tr.inter[l][c]), (l, c)
                noff += nc[off + c]
                ioff += ic[off + c]
            off += n
    finally:
        pb.pb_destroy(ctx)


def test_morton_order_large_and_tied():
    """The stable radix sort of the Morton keys (Section 2.4) on 81920 triangles (320 sort tiles,
    a ragged last scan tile) and on two copies of that surface 2e-4 apart, where most keys tie
    with the key of the element 81920 places later (another sort tile): the order must be the
    keys' order with ties by element index, bit for bit."""
    m = inputs.kirkwood_ball(6, 2.0, 3, 1.5, seed=6)
    V2 = np.vstack([m.verts, m.verts + 2e-4])
    T2 = np.vstack([m.tris, m.tris + len(m.verts)])
    for V, T in ((m.verts, m.tris), (V2, T2)):
        ctx = _ctx(inputs.Mesh(V, T, m.qpos, m.q), leaf_size=64, eta0=0.8, precision=pb.PB_FP64)
        try:
            st, order, *_ = pb.pb_get_tree(ctx, len(T))
        finally:
            pb.pb_destroy(ctx)
        key, _, _ = fmm.morton_keys(fmm.centroids(V, T), V)
        ref = np.lexsort((np.arange(len(T)), key))
        assert np.array_equal(order, ref)
        if len(T) > len(m.tris):
            assert np.count_nonzero(np.diff(key[ref]) == 0) > len(m.tris) // 2  # many ties


def test_all_near_fp64_equals_dense(sphere3):
    m, ph, A = sphere3
    ctx = _ctx(m, leaf_size=16, eta0=1e-6, p=2, precision=pb.PB_FP64)
    try:
        x = inputs.random_density(m.nt, 5)
        y = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
        pb.pb_matvec(ctx, _dev(x), y)
        assert _rel(y.cpu().numpy(), A @ x) < 1e-12
    finally:
        pb.pb_destroy(ctx)


def test_float_float_singular_equals_dense(sphere3):
    # the Sauter-Schwab integrals in float-float reproduce the FP64 oracle's Galerkin matrix
    m, ph, A = sphere3
    ctx = _ctx(m, leaf_size=16, eta0=1e-6, p=2, precision=pb.PB_FP64, singular=pb.PB_SINGULAR_FF)
    try:
        x = inputs.random_density(m.nt, 5)
        y = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
        pb.pb_matvec(ctx, _dev(x), y)
        assert _rel(y.cpu().numpy(), A @ x) < 1e-11
    finally:
        pb.pb_destroy(ctx)


@pytest.mark.parametrize("kappa", [KAP, 2.5])
def test_float_float_singular_matches_fp64_on_molecule(kappa):
    # irregular marching-tetrahedra triangles; kappa = 2.5 takes kappa r past 0.5 (FP64 exp branch)
    from paper_2110_13778_gb300 import molecules

    m = molecules.molecule(40, 4040, 1.0)[0]
    x = _dev(inputs.random_density(m.nt, 6))
    ys = []
    for mode in (pb.PB_SINGULAR_FP64, pb.PB_SINGULAR_FF):
        ctx = _ctx(m, leaf_size=32, eta0=0.7, p=4, kappa=kappa, precision=pb.PB_FP64, singular=mode)
        try:
            y = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
            pb.pb_matvec_part(ctx, x, y, 1)
            ys.append(y.cpu().numpy())
        finally:
            pb.pb_destroy(ctx)
    assert _rel(ys[1], ys[0]) < 1e-11


@pytest.mark.parametrize("p,adaptive", [(4, 0), (6, 0), (8, 0), (3, 1), (5, 0)])
def test_fmm_fp64_matches_oracle_fmm(sphere3, p, adaptive):
    m, ph, A = sphere3
    ctx = _ctx(m, leaf_size=16, eta0=0.8, p=p, adaptive=adaptive, precision=pb.PB_FP64)
    try:
        x = inputs.random_density(m.nt, 9)
        xd = _dev(x)
        y = torch.empty_like(xd)
        pb.pb_matvec(ctx, xd, y)
        tr = fmm.Tree(m.verts, m.tris, leaf_size=16, eta0=0.8)
        yo = fmm.matvec(tr, m.verts, m.tris, x, ph, p, adaptive=bool(adaptive), A=A)
        assert _rel(y.cpu().numpy(), yo) < 1e-10
        # far field alone (no near, no mass)
        yf = torch.empty_like(xd)
        pb.pb_matvec_part(ctx, xd, yf, 2)
        f1, f2 = fmm.far_field(tr, m.verts, m.tris, x, ph, p, adaptive=bool(adaptive))
        assert _rel(yf.cpu().numpy(), np.r_[f1, f2]) < 1e-10
    finally:
        pb.pb_destroy(ctx)


def test_fmm_p8_within_1e4_of_dense(sphere3):
    m, ph, A = sphere3
    for prec in (pb.PB_FP64, pb.PB_MIXED):
        ctx = _ctx(m, leaf_size=16, eta0=0.8, p=8, precision=prec)
        try:
            x = inputs.random_density(m.nt, 11)
            y = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
            pb.pb_matvec(ctx, _dev(x), y)
            assert _rel(y.cpu().numpy(), A @ x) < 1e-4
        finally:
            pb.pb_destroy(ctx)


@pytest.mark.parametrize("p,adaptive", [(4, 0), (6, 0), (8, 0), (10, 0), (5, 0), (3, 1), (2, 0), (7, 0), (9, 0)])
def test_mixed_matches_oracle_fmm(sphere3, p, adaptive):
    # p = 4, 6, 8 run the generated MtL bodies; p = 10, 5, 2, 7, 9 and the adaptive orders
    # (3..6 by level) the generic FP32 recurrence MtL; every order runs its own fixed-order LtP
    m, ph, A = sphere3
    ctx = _ctx(m, leaf_size=16, eta0=0.8, p=p, adaptive=adaptive, precision=pb.PB_MIXED)
    try:
        x = inputs.random_density(m.nt, 13)
        y = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
        pb.pb_matvec(ctx, _dev(x), y)
        tr = fmm.Tree(m.verts, m.tris, leaf_size=16, eta0=0.8)
        yo = fmm.matvec(tr, m.verts, m.tris, x, ph, p, adaptive=bool(adaptive), A=A)
        assert _rel(y.cpu().numpy(), yo) < 2e-5
        yf = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
        pb.pb_matvec_part(ctx, _dev(x), yf, 2)
        f1, f2 = fmm.far_field(tr, m.verts, m.tris, x, ph, p, adaptive=bool(adaptive))
        assert _rel(yf.cpu().numpy(), np.r_[f1, f2]) < 1e-4
    finally:
        pb.pb_destroy(ctx)


def test_rhs_and_energy_match_oracle(sphere3):
    m, ph, A = sphere3
    for prec, tol in ((pb.PB_FP64, 1e-12), (pb.PB_MIXED, 1e-6)):
        ctx = _ctx(m, leaf_size=16, eta0=0.8, p=4, precision=prec)
        try:
            b = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
            pb.pb_rhs(ctx, b)
            bo = dense.rhs(m, ph)
            assert _rel(b.cpu().numpy(), bo) < tol
            x = np.linalg.solve(A, bo)
            E = pb.pb_solvation_energy(ctx, _dev(x))
            Eo = dense.energy(m, ph, x)
            assert abs(E - Eo) < tol * abs(Eo)
        finally:
            pb.pb_destroy(ctx)


def test_block_preconditioner_matches_leaf_blocks(sphere3):
    m, ph, A = sphere3
    ctx = _ctx(m, leaf_size=16, eta0=0.8, p=4, precond=pb.PB_PRECOND_BLOCK)
    try:
        tr = fmm.Tree(m.verts, m.tris, leaf_size=16, eta0=0.8)
        r = inputs.random_density(m.nt, 17)
        z = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
        pb.pb_precond_apply(ctx, _dev(r), z)
        N = m.nt
        zo = np.zeros(2 * N)
        for c in range(tr.nclusters(tr.L)):
            e = tr.order[tr.begin[tr.L][c]:tr.end[tr.L][c]]
            idx = np.r_[e, N + e]
            zo[idx] = np.linalg.solve(A[np.ix_(idx, idx)], r[idx])
        assert _rel(z.cpu().numpy(), zo) < 1e-10
    finally:
        pb.pb_destroy(ctx)


@pytest.mark.parametrize("prec,precond", [(pb.PB_FP64, pb.PB_PRECOND_BLOCK), (pb.PB_MIXED, pb.PB_PRECOND_BLOCK),
                                          (pb.PB_FP64, pb.PB_PRECOND_DIAG), (pb.PB_MIXED, pb.PB_PRECOND_NONE)])
def test_gmres_solution_and_energy(sphere3, prec, precond):
    m, ph, A = sphere3
    ctx = _ctx(m, leaf_size=16, eta0=0.6, p=8, precision=prec, precond=precond)
    try:
        x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
        tol = 1e-8 if prec == pb.PB_FP64 else 1e-6
        info = pb.pb_gmres_solve(ctx, x, tol=tol, max_iter=200, restart=50)
        assert info.status == pb.PB_OK and info.rel_residual < 1.5 * tol
        xo = np.linalg.solve(A, dense.rhs(m, ph))
        assert _rel(x.cpu().numpy(), xo) < 1e-4
        E = pb.pb_solvation_energy(ctx, x)
        Eo = dense.energy(m, ph, xo)
        assert abs(E - Eo) < 1e-4 * abs(Eo)
    finally:
        pb.pb_destroy(ctx)


def test_kirkwood_small_sphere_energy():
    # the 2 A, +1 e Kirkwood sphere at 1280 triangles: oracle parity and the closed form
    m = inputs.kirkwood_centered(3, 2.0, 1.0)
    ph = dense.Phys(1.0, 80.0, KAP, qs=3)
    xo, A, b = dense.solve(m, ph)
    Eo = dense.energy(m, ph, xo)
    ex = kirkwood.centered(1.0, 2.0, 1.0, 80.0, KAP)
    for prec in (pb.PB_FP64, pb.PB_MIXED):
        ctx = _ctx(m, leaf_size=16, eta0=0.8, p=8, precision=prec)
        try:
            x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
            info = pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=100, restart=50)
            assert info.status == pb.PB_OK
            E = pb.pb_solvation_energy(ctx, x)
            assert abs(E - Eo) < 1e-3 * abs(Eo)
            assert abs(E - ex) < 0.015 * abs(ex)
        finally:
            pb.pb_destroy(ctx)


def test_bad_mesh_rejected():
    V, T = inputs.icosphere(1, 1.0)
    prm = pb.params()
    ctx = pb.pb_create(prm)
    try:
        Tb = T.copy()
        Tb[3, 1] = 10_000
        with pytest.raises(pb.PBError) as e:
            pb.pb_mesh_upload(ctx, V, Tb, np.zeros((1, 3)), np.ones(1))
        assert e.value.code == pb.PB_ERR_MESH
        Tz = T.copy()
        Tz[0] = [0, 0, 1]
        with pytest.raises(pb.PBError):
            pb.pb_mesh_upload(ctx, V, Tz, np.zeros((1, 3)), np.ones(1))
        with pytest.raises(pb.PBError) as e:
            pb.pb_build_tree(ctx)
        assert e.value.code == pb.PB_ERR_STATE
    finally:
        pb.pb_destroy(ctx)


def test_tiny_and_ragged_meshes():
    # single-level tree (everything near) and a mesh smaller than one leaf
    for lev, leaf in ((0, 64), (1, 64), (2, 7)):
        V, T = inputs.perturbed_sphere(lev, 3.0, 0.1, seed=lev) if lev else inputs.icosphere(0, 3.0)
        m = inputs.Mesh(V, T, np.zeros((1, 3)), np.ones(1))
        ph = dense.Phys(1.0, 80.0, KAP, qs=3)
        A = dense.assemble(V, T, ph)
        ctx = _ctx(m, leaf_size=leaf, eta0=0.8, p=6, precision=pb.PB_FP64)
        try:
            x = inputs.random_density(m.nt, 2)
            y = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
            pb.pb_matvec(ctx, _dev(x), y)
            tr = fmm.Tree(V, T, leaf_size=leaf, eta0=0.8)
            yo = fmm.matvec(tr, V, T, x, ph, 6, A=A)
            assert _rel(y.cpu().numpy(), yo) < 1e-10
        finally:
            pb.pb_destroy(ctx)
