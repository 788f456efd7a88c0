"""The Cartesian treecode for the solvation energy (Section 2.5: eqMAC, addCluster,
eqsolengformTree) against the oracle's treecode (oracle.fmm.treecode_energy: the same MAC
decisions, FP64) and against the direct sum it approximates. Needs a GPU."""
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
def sphere():
    m = inputs.kirkwood_ball(3, 20.0, 12, 16.0, seed=5)
    ph = dense.Phys(1.0, 80.0, KAP, qs=3)
    x, _, _ = dense.solve(m, ph)
    return m, ph, x


def _ctx(m, precision, p=8, adaptive=0, leaf=16):
    ctx = pb.pb_create(pb.params(eps_in=1.0, eps_out=80.0, kappa=KAP, eta0=0.8, leaf_size=leaf, p=p,
                                 adaptive=adaptive, precision=precision))
    pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
    pb.pb_build_tree(ctx)
    return ctx


def _dev(x):
    return torch.tensor(np.asarray(x), device="cuda", dtype=torch.float64)


@pytest.mark.parametrize("p,theta,adaptive", [(4, 0.5, 0), (8, 0.5, 0), (8, 0.7, 0), (3, 0.6, 1)])
def test_fp64_matches_oracle_treecode(sphere, p, theta, adaptive):
    m, ph, x = sphere
    ctx = _ctx(m, pb.PB_FP64, p, adaptive)
    try:
        E = pb.pb_solvation_energy_treecode(ctx, _dev(x), theta)
        tr = fmm.Tree(m.verts, m.tris, leaf_size=16, eta0=0.8)
        Eo = fmm.treecode_energy(tr, m, x, ph, p, theta, adaptive=bool(adaptive))
        assert abs(E - Eo) < 1e-10 * abs(Eo), (E, Eo)
        # and the approximation it makes: near the direct sum, closer at higher order
        Ed = dense.energy(m, ph, x)
        assert abs(E - Ed) < (1e-3 if p < 6 else 5e-5) * abs(Ed)
    finally:
        pb.pb_destroy(ctx)


def test_small_theta_is_the_direct_sum(sphere):
    m, ph, x = sphere
    for prec, tol in ((pb.PB_FP64, 1e-12), (pb.PB_MIXED, 1e-6)):
        ctx = _ctx(m, prec)
        try:
            xd = _dev(x)
            E = pb.pb_solvation_energy_treecode(ctx, xd, 1e-6)
            Ed = pb.pb_solvation_energy(ctx, xd)
            assert abs(E - Ed) < tol * abs(Ed)
        finally:
            pb.pb_destroy(ctx)


def test_mixed_matches_oracle_treecode(sphere):
    m, ph, x = sphere
    ctx = _ctx(m, pb.PB_MIXED, 6)
    try:
        E = pb.pb_solvation_energy_treecode(ctx, _dev(x), 0.5)
        tr = fmm.Tree(m.verts, m.tris, leaf_size=16, eta0=0.8)
        Eo = fmm.treecode_energy(tr, m, x, ph, 6, 0.5)
        assert abs(E - Eo) < 2e-6 * abs(Eo)
    finally:
        pb.pb_destroy(ctx)


def test_far_charges_take_the_root_series_and_single_leaf_tree():
    # charges far outside the surface: the root satisfies the MAC; and a mesh of one leaf
    V, T = inputs.icosphere(2, 3.0)
    qp = np.array([[60.0, 10.0, -5.0], [-40.0, 55.0, 20.0], [0.5, 0.2, -0.3]])
    m = inputs.Mesh(V, T, qp, np.array([1.0, -0.5, 0.7]))
    ph = dense.Phys(1.0, 80.0, KAP, qs=3)
    x = inputs.random_density(m.nt, 4)
    for leaf in (16, 1000):
        ctx = _ctx(m, pb.PB_FP64, 6, leaf=leaf)
        try:
            E = pb.pb_solvation_energy_treecode(ctx, _dev(x), 0.5)
            tr = fmm.Tree(m.verts, m.tris, leaf_size=leaf, eta0=0.8)
            assert (tr.L == 0) == (leaf == 1000)
            Eo = fmm.treecode_energy(tr, m, x, ph, 6, 0.5)
            assert abs(E - Eo) < 1e-10 * abs(Eo), (leaf, E, Eo)
        finally:
            pb.pb_destroy(ctx)


def test_molecule_treecode_near_direct():
    m = molecules.molecule(60, 3060, 1.0)[0]
    for prec in (pb.PB_FP64, pb.PB_MIXED):
        ctx = _ctx(m, prec, 8, leaf=64)
        try:
            x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
            pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=200, restart=50)
            Ed = pb.pb_solvation_energy(ctx, x)
            E = pb.pb_solvation_energy_treecode(ctx, x, 0.5)
            assert abs(E - Ed) < 2e-5 * abs(Ed)
        finally:
            pb.pb_destroy(ctx)
