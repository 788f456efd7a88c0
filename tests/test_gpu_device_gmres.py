"""The device-driven GMRES (one CUDA graph launch per solve: conditional WHILE nodes for the
Arnoldi steps and the restart cycles, every stopping decision taken on the device) against the
host-driven loop it replaces (still taken when per-phase timing is enabled): the same
iterations, products, residuals and solutions, for one and for several right-hand sides, with
restarts, given starts and the iteration cap. Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def _ctx(m, precision=pb.PB_MIXED, precond=pb.PB_PRECOND_BLOCK):
    ctx = pb.pb_create(pb.params(eps_in=1.0, eps_out=80.0, kappa=KAP, eta0=0.7, leaf_size=32, p=6,
                                 precision=precision, precond=precond))
    pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
    pb.pb_build_tree(ctx)
    return ctx


def _solve(ctx, n, timing, x0=None, **kw):
    pb.pb_set_timing(ctx, 1 if timing else 0)
    x = torch.zeros(2 * n, device="cuda", dtype=torch.float64) if x0 is None else x0.clone()
    g0 = pb.pb_get_graph_launches(ctx)
    info = pb.pb_gmres_solve(ctx, x, use_x0=x0 is not None, raise_on_fail=False, **kw)
    g1 = pb.pb_get_graph_launches(ctx)
    pb.pb_set_timing(ctx, 0)
    return x, info, g1 - g0


def _same(a, b, exact=True):
    # FP64 products are reproducible to rounding; the mixed near field sums FP32 partials
    # through shared-memory atomics, so two mixed runs agree to FP32 rounding only: the
    # iteration count may move by one and a residual near its FP32 floor by some per cent
    assert a.status == b.status
    if exact:
        assert a.iterations == b.iterations
        assert a.matvecs == b.matvecs
        assert abs(a.rel_residual - b.rel_residual) <= 1e-6 * max(abs(b.rel_residual), 1e-14)
        assert abs(a.initial_residual - b.initial_residual) <= 1e-9 * abs(b.initial_residual)
    else:
        assert abs(a.iterations - b.iterations) <= 1
        assert abs(a.rel_residual - b.rel_residual) <= 0.5 * b.rel_residual + 1e-12
        assert abs(a.initial_residual - b.initial_residual) <= 1e-5 * abs(b.initial_residual)


@pytest.fixture(scope="module")
def mol():
    return molecules.molecule(40, 4040, 1.0)[0]


@pytest.mark.parametrize("precision", [pb.PB_MIXED, pb.PB_FP64])
@pytest.mark.parametrize("restart,max_iter,tol", [(50, 200, 1e-8), (3, 200, 1e-8), (4, 6, 1e-10)])
def test_single_solve_matches_host_loop(mol, precision, restart, max_iter, tol):
    if precision == pb.PB_MIXED and max_iter > 6:
        tol = 1e-6  # the FP32 product's rounding puts the true residual's floor near 1e-7
    ctx = _ctx(mol, precision)
    try:
        n = mol.nt
        xh, ih, gh = _solve(ctx, n, True, tol=tol, max_iter=max_iter, restart=restart)
        xd, idv, gd = _solve(ctx, n, False, tol=tol, max_iter=max_iter, restart=restart)
        assert gh == 0 and gd == 1  # the device-driven solve is one graph launch
        exact = precision == pb.PB_FP64
        _same(idv, ih, exact)
        if max_iter == 6:
            assert idv.status == pb.PB_ERR_NOT_CONVERGED and idv.iterations == 6
        else:
            assert idv.status == pb.PB_OK and idv.rel_residual < 2 * tol
        d = (xd - xh).norm().item() / xh.norm().item()
        assert d < (1e-10 if exact else 1e-5)
        # the cached graph is replayed by the next solve of the same shape
        xd2, idv2, gd2 = _solve(ctx, n, False, tol=tol, max_iter=max_iter, restart=restart)
        assert gd2 == 1
        _same(idv2, idv, exact)
        assert (xd2 - xd).norm().item() <= (1e-12 if exact else 1e-5) * xd.norm().item()
    finally:
        pb.pb_destroy(ctx)


def test_given_start_matches_host_loop(mol):
    ctx = _ctx(mol, pb.PB_FP64)
    try:
        n = mol.nt
        x, _, _ = _solve(ctx, n, False, tol=1e-8, max_iter=200, restart=50)
        start = x * (1.0 + 0.05 * torch.sin(torch.arange(2 * n, device="cuda", dtype=torch.float64)))
        xh, ih, _ = _solve(ctx, n, True, x0=start, tol=1e-8, max_iter=200, restart=50)
        xd, idv, gd = _solve(ctx, n, False, x0=start, tol=1e-8, max_iter=200, restart=50)
        assert gd == 1
        _same(idv, ih)
        assert idv.initial_residual < 0.2 and idv.matvecs == idv.iterations + 2
        assert (xd - xh).norm().item() / xh.norm().item() < 1e-10
    finally:
        pb.pb_destroy(ctx)


def test_rebuild_recaptures():
    # a new build (new buffers) must not replay a graph that points at the old ones
    m1 = inputs.kirkwood_ball(3, 2.0, 5, 1.5, seed=3)
    ctx = _ctx(m1, pb.PB_FP64)
    try:
        n = m1.nt
        x1, i1, _ = _solve(ctx, n, False, tol=1e-9, max_iter=100, restart=30)
        E1 = pb.pb_solvation_energy(ctx, x1)
        for _ in range(2):
            pb.pb_build_tree(ctx)
            x2, i2, g = _solve(ctx, n, False, tol=1e-9, max_iter=100, restart=30)
            assert g == 1 and i2.iterations == i1.iterations
            assert abs(pb.pb_solvation_energy(ctx, x2) - E1) < 1e-12 * abs(E1)
        V2, T2 = inputs.perturbed_sphere(3, 2.0, 0.05, seed=8)
        m2 = inputs.Mesh(V2, T2, m1.qpos, m1.q)
        pb.pb_mesh_upload(ctx, m2.verts, m2.tris, m2.qpos, m2.q)
        pb.pb_build_tree(ctx)
        xd, idv, _ = _solve(ctx, m2.nt, False, tol=1e-9, max_iter=100, restart=30)
        xh, ih, _ = _solve(ctx, m2.nt, True, tol=1e-9, max_iter=100, restart=30)
        _same(idv, ih)
    finally:
        pb.pb_destroy(ctx)


@pytest.mark.parametrize("nstates,precision", [(6, pb.PB_FP64), (18, pb.PB_FP64), (18, pb.PB_MIXED)])
def test_batched_states_match_host_loop(mol, nstates, precision):
    rng = np.random.default_rng(7)
    Q = np.repeat(mol.q[None, :], nstates, axis=0)
    for s in range(1, nstates):
        flip = rng.random(mol.nc) < 0.1
        Q[s, flip] = -Q[s, flip]
    ctx = _ctx(mol, precision)
    exact = precision == pb.PB_FP64
    try:
        n2 = 2 * mol.nt
        Xh = torch.empty((nstates, n2), device="cuda", dtype=torch.float64)
        Xd = torch.empty_like(Xh)
        pb.pb_set_timing(ctx, 1)
        Eh, ih = pb.pb_solve_states(ctx, Q, Xh, tol=1e-8, max_iter=200, restart=50, warm=2)
        pb.pb_set_timing(ctx, 0)
        g0 = pb.pb_get_graph_launches(ctx)
        Ed, idv = pb.pb_solve_states(ctx, Q, Xd, tol=1e-8, max_iter=200, restart=50, warm=2)
        # state 0 alone, then the others as one batch (up to 64 per launch)
        assert pb.pb_get_graph_launches(ctx) - g0 == 2
        # (the device path's update applies the block inverses to all states in one launch,
        # the host loop state by state: the same arithmetic up to rounding order)
        for a, b in zip(idv, ih):
            assert a.status == b.status == pb.PB_OK
            _same(a, b, exact)
        assert np.allclose(Ed, Eh, rtol=1e-10 if exact else 1e-6, atol=0)
        assert (Xd - Xh).norm().item() / Xh.norm().item() < (1e-9 if exact else 1e-5)
        # and every state against its own single solve from zero
        for s in (0, nstates - 1):
            pb.pb_set_charges(ctx, Q[s])
            x = torch.zeros(n2, device="cuda", dtype=torch.float64)
            pb.pb_gmres_solve(ctx, x, tol=1e-8, max_iter=200, restart=50)
            E = pb.pb_solvation_energy(ctx, x)
            assert abs(E - Ed[s]) < 1e-6 * abs(E)
    finally:
        pb.pb_destroy(ctx)
