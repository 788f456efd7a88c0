"""Failure paths of the C ABI, made on the host (no GPU fault): a solve that runs out of
iterations, a residual that overflows, a non-finite learned start (which falls back to the
zero start), non-finite uploads and calls out of order. Needs a GPU for the solver calls."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2110_13778_gb300 import inputs, pb  # noqa: E402

pytestmark = pytest.mark.gpu

KAP = 0.1257


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_13778_gb300 import build

    build.build()
    pb.lib()


@pytest.fixture()
def sphere():
    m = inputs.kirkwood_ball(3, 2.0, 5, 1.5, seed=3)
    ctx = pb.pb_create(pb.params(eps_in=1.0, eps_out=80.0, kappa=KAP, eta0=0.8, leaf_size=16, p=6,
                                 precision=pb.PB_MIXED, precond=pb.PB_PRECOND_NONE))
    pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
    pb.pb_build_tree(ctx)
    yield m, ctx
    pb.pb_destroy(ctx)


def test_max_iter_gives_not_converged(sphere):
    m, ctx = sphere
    x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
    info = pb.pb_gmres_solve(ctx, x, tol=1e-12, max_iter=2, restart=50, raise_on_fail=False)
    assert info.status == pb.PB_ERR_NOT_CONVERGED
    assert info.iterations == 2
    assert info.matvecs == 3  # two Arnoldi products + the true residual (zero start: none first)
    assert np.isfinite(info.rel_residual) and 1e-12 < info.rel_residual < 1.0
    with pytest.raises(pb.PBError) as e:
        pb.pb_gmres_solve(ctx, x, tol=1e-12, max_iter=2, restart=50)
    assert e.value.code == pb.PB_ERR_NOT_CONVERGED
    # the context stays usable
    info = pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=100, restart=50)
    assert info.status == pb.PB_OK


def test_overflowing_residual_gives_nonfinite():
    # finite charges so large that ||b||^2 overflows: the residual ratio is not finite
    m = inputs.kirkwood_ball(2, 2.0, 3, 1.5, seed=4)
    q = np.full(m.nc, 1e300)
    ctx = pb.pb_create(pb.params(eps_in=1.0, eps_out=80.0, kappa=KAP, eta0=0.8, leaf_size=16, p=4))
    try:
        pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, q)
        pb.pb_build_tree(ctx)
        x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=20, restart=10, raise_on_fail=False)
        assert info.status == pb.PB_ERR_NONFINITE
    finally:
        pb.pb_destroy(ctx)


def test_nonfinite_learned_start_falls_back_to_zero(sphere):
    m, ctx = sphere
    x0 = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
    ref = pb.pb_gmres_solve(ctx, x0, tol=1e-8, max_iter=100, restart=50)
    E0 = pb.pb_solvation_energy(ctx, x0)
    for bad in (float("nan"), float("inf")):
        x = torch.full((2 * m.nt,), bad, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-8, max_iter=100, restart=50, use_x0=True)
        assert info.status == pb.PB_OK
        assert info.iterations == ref.iterations
        assert info.matvecs == ref.matvecs + 1  # the product of the rejected start
        assert torch.isfinite(x).all()
        assert abs(pb.pb_solvation_energy(ctx, x) - E0) < 1e-12 * abs(E0)
    # a start pointing the wrong way (no positive least-squares factor) is dropped too
    x = -x0.clone()
    info = pb.pb_gmres_solve(ctx, x, tol=1e-8, max_iter=100, restart=50, use_x0=True)
    assert info.status == pb.PB_OK and info.iterations == ref.iterations


def test_nonfinite_uploads_rejected():
    V, T = inputs.icosphere(1, 2.0)
    ctx = pb.pb_create(pb.params())
    try:
        for qpos, q in ((np.zeros((1, 3)), np.array([np.nan])), (np.array([[np.inf, 0, 0]]), np.ones(1))):
            with pytest.raises(pb.PBError) as e:
                pb.pb_mesh_upload(ctx, V, T, qpos, q)
            assert e.value.code == pb.PB_ERR_MESH
        Vb = V.copy()
        Vb[2, 1] = np.nan
        with pytest.raises(pb.PBError) as e:
            pb.pb_mesh_upload(ctx, Vb, T, np.zeros((1, 3)), np.ones(1))
        assert e.value.code == pb.PB_ERR_MESH
        pb.pb_mesh_upload(ctx, V, T, np.zeros((1, 3)), np.ones(1))
        with pytest.raises(pb.PBError) as e:
            pb.pb_set_charges(ctx, np.array([np.nan]))
        assert e.value.code == pb.PB_ERR_MESH
    finally:
        pb.pb_destroy(ctx)


def test_calls_out_of_order():
    V, T = inputs.icosphere(1, 2.0)
    ctx = pb.pb_create(pb.params())
    try:
        x = torch.zeros(2 * T.shape[0], device="cuda", dtype=torch.float64)
        y = torch.empty_like(x)
        with pytest.raises(pb.PBError) as e:
            pb.pb_build_tree(ctx)
        assert e.value.code == pb.PB_ERR_STATE
        pb.pb_mesh_upload(ctx, V, T, np.zeros((1, 3)), np.ones(1))
        with pytest.raises(pb.PBError) as e:
            pb.pb_matvec(ctx, x, y)
        assert e.value.code == pb.PB_ERR_STATE
        with pytest.raises(pb.PBError) as e:
            pb.pb_gmres_solve(ctx, x)
        assert e.value.code == pb.PB_ERR_STATE
    finally:
        pb.pb_destroy(ctx)
