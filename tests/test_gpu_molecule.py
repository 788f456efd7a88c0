"""Protein-like molecular surfaces (marching-tetrahedra Gaussian isosurface of a self-avoiding
walk) and batched charge states, CUDA path against the oracle. Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, fmm  # noqa: E402
from paper_2110_13778_gb300 import inputs, molecules, pb  # noqa: E402

pytestmark = pytest.mark.gpu

KAP = 0.1257


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_13778_gb300 import build

    build.build()
    pb.lib()


@pytest.fixture(scope="module")
def mol():
    m, rad = molecules.molecule(40, 4040, 1.0)
    ph = dense.Phys(1.0, 80.0, KAP, qs=3)
    A = dense.assemble(m.verts, m.tris, ph)
    return m, ph, A


def _ctx(m, **kw):
    ctx = pb.pb_create(pb.params(**kw))
    pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
    pb.pb_build_tree(ctx)
    return ctx


def _leaf_blocks(tr, bmax=96):
    """Preconditioner blocks: the leaves, a leaf above bmax elements cut into nearly equal
    consecutive (Morton-ordered) parts of at most bmax elements."""
    out = []
    for c in range(tr.nclusters(tr.L)):
        e = tr.order[tr.begin[tr.L][c]:tr.end[tr.L][c]]
        parts = (len(e) + bmax - 1) // bmax
        base, extra = divmod(len(e), parts)
        s0 = 0
        for q in range(parts):
            n = base + (1 if q < extra else 0)
            out.append(e[s0:s0 + n])
            s0 += n
    return out


@pytest.mark.parametrize("prec,leaf", [(pb.PB_MIXED, 24), (pb.PB_MIXED, 48), (pb.PB_FP64, 24)])
def test_block_preconditioner_all_size_classes(mol, prec, leaf):
    # block inverses of every register-tile class (order <= 64, <= 128, <= 192 under mixed
    # precision) against FP64 solves with the oracle's diagonal blocks of the dense matrix
    m, ph, A = mol
    ctx = _ctx(m, leaf_size=leaf, eta0=0.8, p=4, precision=prec, precond=pb.PB_PRECOND_BLOCK)
    try:
        tr = fmm.Tree(m.verts, m.tris, leaf_size=leaf, eta0=0.8)
        blocks = _leaf_blocks(tr)
        classes = {0 if 2 * len(e) <= 64 else 1 if 2 * len(e) <= 128 else 2 for e in blocks}
        assert classes == {0, 1, 2}  # the molecule's leaves span all three
        st = pb.pb_get_tree_stats(ctx)
        assert st["pc_blocks"] == len(blocks)
        assert st["pc_max"] == 2 * max(len(e) for e in blocks)
        r = inputs.random_density(m.nt, 29)
        z = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
        pb.pb_precond_apply(ctx, torch.tensor(r, device="cuda", dtype=torch.float64), z)
        N = m.nt
        zo = np.zeros(2 * N)
        for e in blocks:
            idx = np.r_[e, N + e]
            zo[idx] = np.linalg.solve(A[np.ix_(idx, idx)], r[idx])
        d = float(np.linalg.norm(z.cpu().numpy() - zo) / np.linalg.norm(zo))
        # FP32 entries and Gauss-Jordan lose a few digits against FP64
        assert d < (1e-10 if prec == pb.PB_FP64 else 2e-4), d
    finally:
        pb.pb_destroy(ctx)


@pytest.mark.parametrize("prec", [pb.PB_FP64, pb.PB_MIXED])
def test_molecule_solve_matches_oracle(mol, prec):
    m, ph, A = mol
    xo = np.linalg.solve(A, dense.rhs(m, ph))
    Eo = dense.energy(m, ph, xo)
    ctx = _ctx(m, leaf_size=32, eta0=0.7, p=8, precision=prec)
    try:
        x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=300, restart=50)
        assert info.status == pb.PB_OK
        E = pb.pb_solvation_energy(ctx, x)
        assert abs(E - Eo) < 1e-3 * abs(Eo), (E, Eo)
        xn = x.cpu().numpy()
        assert np.linalg.norm(xn - xo) / np.linalg.norm(xo) < 5e-3
    finally:
        pb.pb_destroy(ctx)


def test_charge_states_batch_matches_oracle(mol):
    m, ph, A = mol
    rng = np.random.default_rng(7)
    states = []
    for s in range(4):
        q = m.q.copy()
        flip = rng.random(q.size) < 0.05
        q[flip] = -q[flip]
        states.append(q)
    Q = np.array(states)
    ctx = _ctx(m, leaf_size=32, eta0=0.7, p=8, precision=pb.PB_MIXED)
    try:
        X = torch.zeros((len(states), 2 * m.nt), device="cuda", dtype=torch.float64)
        E, infos = pb.pb_solve_states(ctx, Q, X, tol=1e-6, max_iter=300, restart=50, warm=True)
        assert all(i.status == pb.PB_OK for i in infos)
        B = np.stack([dense.rhs(dense_mesh(m, q), ph) for q in states], axis=1)
        Xo = np.linalg.solve(A, B)
        for s, q in enumerate(states):
            Eo = dense.energy(dense_mesh(m, q), ph, Xo[:, s])
            assert abs(E[s] - Eo) < 1e-3 * abs(Eo), (s, E[s], Eo)
        # the warm start from the previous state saves iterations
        assert infos[1].iterations <= infos[0].iterations
    finally:
        pb.pb_destroy(ctx)


def dense_mesh(m, q):
    from paper_2110_13778_gb300.inputs import Mesh

    return Mesh(m.verts, m.tris, m.qpos, q)


@pytest.mark.parametrize("prec,nrhs", [(pb.PB_FP64, 1), (pb.PB_MIXED, 1), (pb.PB_MIXED, 4)])
def test_autotune_picks_an_accurate_configuration(mol, prec, nrhs):
    m, ph, A = mol
    xo = np.linalg.solve(A, dense.rhs(m, ph))
    Eo = dense.energy(m, ph, xo)
    ctx = pb.pb_create(pb.params(eta0=0.7, leaf_size=64, p=8, precision=prec))
    try:
        pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
        with pytest.raises(pb.PBError):
            pb.pb_autotune(ctx, tol=1e-4, matvecs_per_solve=10, nrhs=0)
        r = pb.pb_autotune(ctx, tol=1e-4, matvecs_per_solve=10, nrhs=nrhs)
        assert r["met_tolerance"] == 1 and r["rel_err"] <= 1e-4
        assert r["leaf_size"] in (32, 48, 64, 96, 128) and r["p"] in (4, 6, 8)
        assert r["tried"] >= 5 and r["matvec_ms"] > 0
        # per-level orders: never above the uniform choice, never below 4, and the context's
        # build uses them
        st = pb.pb_get_tree_stats(ctx)
        L = st["levels"]
        assert list(st["order"][:L + 1]) == r["order"][:L + 1]
        assert all(4 <= o <= r["p"] for o in r["order"][1:L + 1])
        pb.pb_build_tree(ctx)
        assert list(pb.pb_get_tree_stats(ctx)["order"][:L + 1]) == r["order"][:L + 1]
        # the context is left built with the choice and solves to the oracle's energy
        x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=300, restart=50)
        assert info.status == pb.PB_OK
        E = pb.pb_solvation_energy(ctx, x)
        assert abs(E - Eo) < 1e-3 * abs(Eo), (E, Eo)
    finally:
        pb.pb_destroy(ctx)


@pytest.mark.parametrize("prec,nr", [(pb.PB_FP64, 3), (pb.PB_MIXED, 5), (pb.PB_MIXED, 19)])
def test_matvec_multi_matches_single_products(mol, prec, nr):
    # 19 right-hand sides take the 16-, 2- and 1-wide near-field kernels
    m, ph, A = mol
    ctx = _ctx(m, leaf_size=32, eta0=0.7, p=6, precision=prec)
    try:
        rng = np.random.default_rng(nr)
        X = torch.tensor(rng.standard_normal((nr, 2 * m.nt)), device="cuda", dtype=torch.float64)
        Y = torch.empty_like(X)
        pb.pb_matvec_multi(ctx, X, Y)
        y1 = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
        for q in range(nr):
            pb.pb_matvec(ctx, X[q].contiguous(), y1)
            d = float((Y[q] - y1).norm() / y1.norm())
            # FP64 runs the same arithmetic per vector; mixed regroups the FP32 near-field sums
            assert d < (1e-14 if prec == pb.PB_FP64 else 1e-6), (q, d)
    finally:
        pb.pb_destroy(ctx)


@pytest.mark.parametrize("prec", [pb.PB_FP64, pb.PB_MIXED])
def test_batched_charge_states_match_sequential(mol, prec):
    m, ph, A = mol
    rng = np.random.default_rng(11)
    states = []
    for s in range(6):
        q = m.q.copy()
        flip = rng.random(q.size) < 0.05
        q[flip] = -q[flip]
        states.append(q)
    Q = np.array(states)
    res = {}
    for mode in (1, 2):
        ctx = _ctx(m, leaf_size=32, eta0=0.7, p=8, precision=prec)
        try:
            X = torch.zeros((len(states), 2 * m.nt), device="cuda", dtype=torch.float64)
            E, infos = pb.pb_solve_states(ctx, Q, X, tol=1e-6, max_iter=300, restart=50, warm=mode)
            assert all(i.status == pb.PB_OK for i in infos)
            assert all(i.rel_residual <= 1.5e-6 for i in infos)
            res[mode] = (E, X.cpu().numpy(), infos)
            # every solve is one CUDA-graph launch: one per state sequentially (mode 1), state 0
            # and then one launch for the other five (mode 2)
            assert pb.pb_get_graph_launches(ctx) == (len(states) if mode == 1 else 2)
        finally:
            pb.pb_destroy(ctx)
    Es, Xs, _ = res[1]
    Eb, Xb, ib = res[2]
    for s in range(len(states)):
        assert abs(Eb[s] - Es[s]) < 1e-5 * abs(Es[s]), (s, Eb[s], Es[s])
        assert np.linalg.norm(Xb[s] - Xs[s]) / np.linalg.norm(Xs[s]) < 1e-4
    # the batched states start from state 0's solution where that beats a zero start
    assert all(i.initial_residual <= 1.0 for i in ib[1:])
    Eo = dense.energy(dense_mesh(m, states[3]), ph, np.linalg.solve(A, dense.rhs(dense_mesh(m, states[3]), ph)))
    assert abs(Eb[3] - Eo) < 1e-3 * abs(Eo)


def test_many_batched_states_match_single_state_calls(mol):
    # 18 states: state 0 alone, then 17 in lockstep, whose right-hand sides and energies are
    # formed 16 states per launch (a group of 16 and a group of 1)
    m, ph, A = mol
    rng = np.random.default_rng(23)
    Q = np.repeat(m.q[None, :], 18, axis=0)
    for s in range(1, 18):
        flip = rng.random(m.q.size) < 0.05
        Q[s, flip] = -Q[s, flip]
    ctx = _ctx(m, leaf_size=32, eta0=0.7, p=8, precision=pb.PB_MIXED)
    try:
        X = torch.zeros((18, 2 * m.nt), device="cuda", dtype=torch.float64)
        E, infos = pb.pb_solve_states(ctx, Q, X, tol=1e-6, max_iter=300, restart=50, warm=2)
        assert all(i.status == pb.PB_OK and i.rel_residual <= 1.5e-6 for i in infos)
        for s in (1, 9, 16, 17):
            pb.pb_set_charges(ctx, Q[s])
            # the batched energy against the single-state energy of the same solution
            Es = pb.pb_solvation_energy(ctx, X[s].contiguous())
            assert abs(E[s] - Es) < 1e-7 * abs(Es), (s, E[s], Es)
            # and the batched solution against a single solve of that state
            x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
            info = pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=300, restart=50)
            assert info.status == pb.PB_OK
            d = float((X[s] - x).norm() / x.norm())
            assert d < 1e-4, (s, d)
    finally:
        pb.pb_destroy(ctx)


def test_multi_entry_points_reject_bad_sizes(mol):
    m, ph, A = mol
    ctx = _ctx(m, leaf_size=32, eta0=0.7, p=6, precision=pb.PB_MIXED)
    try:
        X = torch.zeros((pb.PB_MAX_RHS + 1, 2 * m.nt), device="cuda", dtype=torch.float64)
        with pytest.raises(pb.PBError):
            pb.pb_matvec_multi(ctx, X, torch.empty_like(X))
        Q = np.repeat(m.q[None, :], 2, axis=0)
        with pytest.raises(pb.PBError):
            pb.lib().pb_solve_states  # the binding forwards warm unchanged only for 0/1/2
            rc = pb.lib().pb_solve_states(ctx, Q.ctypes.data_as(pb.ctypes.POINTER(pb.ctypes.c_double)), 2,
                                          pb._ptr(X[:2].contiguous()), None, 1e-6, 100, 50, 3, None)
            pb._check(ctx, rc)
        # one vector through the multi-vector entry point is the plain product
        x = X[:1].contiguous().normal_()
        y1 = torch.empty_like(x)
        pb.pb_matvec_multi(ctx, x, y1)
        y = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
        pb.pb_matvec(ctx, x[0].contiguous(), y)
        assert float((y1[0] - y).norm() / y.norm()) < 1e-12
    finally:
        pb.pb_destroy(ctx)
