"""Parity at the benchmark's full sizes, in the configuration bench.py times, on outputs the
oracle computes one by one: sampled rows of the product (dense Galerkin rows, oracle.dense)
and the residual of the GPU solution on sampled rows. Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense  # noqa: E402
from paper_2110_13778_gb300 import inputs, molecules, pb  # noqa: E402

pytestmark = pytest.mark.gpu

KAP = 0.1257
PH = dense.Phys(1.0, 80.0, KAP, qs=3)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_13778_gb300 import build

    build.build()
    pb.lib()


def _bench_ctx(mesh, precision):
    prm = pb.params(eps_in=1.0, eps_out=80.0, kappa=KAP, eta0=0.8, leaf_size=64, p=8, qs=3, precision=precision,
                    precond=pb.PB_PRECOND_BLOCK)
    ctx = pb.pb_create(prm)
    pb.pb_mesh_upload(ctx, mesh.verts, mesh.tris, mesh.qpos, mesh.q)
    pb.pb_build_tree(ctx)
    return ctx


def _sampled_rows(mesh, ctx, nrows, seed):
    rng = np.random.default_rng(seed)
    x = inputs.random_density(mesh.nt, seed)
    y = torch.empty(2 * mesh.nt, device="cuda", dtype=torch.float64)
    pb.pb_matvec(ctx, torch.tensor(x, device="cuda", dtype=torch.float64), y)
    rows = np.sort(rng.choice(mesh.nt, nrows, replace=False))
    y1, y2 = dense.rows_matvec(mesh.verts, mesh.tris, PH, rows, x)
    yg = y.cpu().numpy()
    ref = np.concatenate([y1, y2])
    got = np.concatenate([yg[rows], yg[mesh.nt + rows]])
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def sphere6():
    # the default benchmark workload: level 6 (81920 triangles), radius 20, 50 charges
    return inputs.kirkwood_ball(6, 20.0, 50, 16.0, 2000)


@pytest.mark.parametrize("prec", [pb.PB_MIXED, pb.PB_FP64])
def test_sphere_level6_sampled_rows(sphere6, prec):
    ctx = _bench_ctx(sphere6, prec)
    try:
        assert _sampled_rows(sphere6, ctx, 192, 61) < 1e-4
    finally:
        pb.pb_destroy(ctx)


def test_sphere_level6_solution_residual_on_sampled_rows(sphere6):
    m = sphere6
    ctx = _bench_ctx(m, pb.PB_MIXED)
    try:
        x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=300, restart=50)
        assert info.status == pb.PB_OK
        xs = x.cpu().numpy()
        rows = np.sort(np.random.default_rng(62).choice(m.nt, 128, replace=False))
        y1, y2 = dense.rows_matvec(m.verts, m.tris, PH, rows, xs)
        b = dense.rhs(m, PH)
        r = np.concatenate([b[rows] - y1, b[m.nt + rows] - y2])
        bb = np.concatenate([b[rows], b[m.nt + rows]])
        # GMRES stops at 1e-6 on the FMM operator; the dense operator differs by the FMM error
        assert np.linalg.norm(r) / np.linalg.norm(bb) < 2e-4
    finally:
        pb.pb_destroy(ctx)


def test_molecule_2000_atoms_sampled_rows():
    # the molecule workload: 2000-atom walk on a 0.9 A grid (~206k triangles)
    m = molecules.molecule(2000, 5000, 0.9)[0]
    assert m.nt > 150000
    ctx = _bench_ctx(m, pb.PB_MIXED)
    try:
        assert _sampled_rows(m, ctx, 128, 63) < 1e-4
    finally:
        pb.pb_destroy(ctx)


@pytest.fixture(scope="module")
def molecule20k():
    # the default benchmark workload: a 20000-atom walk on a 0.9 A grid, short edges collapsed
    # (~1.8M triangles)
    return molecules.molecule(20000, 23000, 0.9, clean=True)[0]


def test_molecule_20000_atoms_sampled_rows(molecule20k):
    m = molecule20k
    assert m.nt > 1_500_000
    ctx = _bench_ctx(m, pb.PB_MIXED)
    try:
        assert _sampled_rows(m, ctx, 48, 64) < 1e-4
    finally:
        pb.pb_destroy(ctx)


def test_molecule_20000_atoms_solve_and_treecode(molecule20k):
    # the benchmark's solve converges on the full molecule; its solution satisfies sampled rows
    # of the dense Galerkin system to the FMM's accuracy; the treecode energy matches the
    # direct sum
    m = molecule20k
    ctx = _bench_ctx(m, pb.PB_MIXED)
    try:
        x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=500, restart=50)
        assert info.status == pb.PB_OK
        xs = x.cpu().numpy()
        rows = np.sort(np.random.default_rng(65).choice(m.nt, 32, replace=False))
        y1, y2 = dense.rows_matvec(m.verts, m.tris, PH, rows, xs)
        # each right-hand-side row depends on its own element only: the oracle's rows from the
        # sub-mesh of the sampled elements
        sub = inputs.Mesh(m.verts, m.tris[rows], m.qpos, m.q)
        bs = dense.rhs(sub, PH)
        r = np.concatenate([bs[:len(rows)] - y1, bs[len(rows):] - y2])
        bb = bs
        assert np.linalg.norm(r) / np.linalg.norm(bb) < 1e-3
        E = pb.pb_solvation_energy(ctx, x)
        Et = pb.pb_solvation_energy_treecode(ctx, x, 0.5)
        assert abs(Et - E) < 1e-5 * abs(E)
    finally:
        pb.pb_destroy(ctx)
