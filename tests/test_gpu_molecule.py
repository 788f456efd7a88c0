"""Protein-like molecular surfaces (marching-tetrahedra Gaussian isosurface of a self-avoiding
walk) and batched charge states, CUDA path against the oracle. Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense  # noqa: E402
from paper_2110_13778_gb300 import molecules, pb  # noqa: E402

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


@pytest.mark.parametrize("prec", [pb.PB_FP64, pb.PB_MIXED])
def test_autotune_picks_an_accurate_configuration(mol, prec):
    m, ph, A = mol
    xo = np.linalg.solve(A, dense.rhs(m, ph))
    Eo = dense.energy(m, ph, xo)
    ctx = pb.pb_create(pb.params(eta0=0.7, leaf_size=64, p=8, precision=prec))
    try:
        pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
        r = pb.pb_autotune(ctx, tol=1e-4, matvecs_per_solve=10)
        assert r["met_tolerance"] == 1 and r["rel_err"] <= 1e-4
        assert r["leaf_size"] in (32, 48, 64, 96, 128) and r["p"] in (4, 6, 8)
        assert r["tried"] >= 5 and r["matvec_ms"] > 0
        st = pb.pb_get_tree_stats(ctx)
        assert all(o == r["p"] for o in st["order"][1:])
        # the context is left built with the choice and solves to the oracle's energy
        x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=300, restart=50)
        assert info.status == pb.PB_OK
        E = pb.pb_solvation_energy(ctx, x)
        assert abs(E - Eo) < 1e-3 * abs(Eo), (E, Eo)
    finally:
        pb.pb_destroy(ctx)
