"""The piecewise-linear basis (continuous hat functions, Section 2.3) on the GPU against the
piecewise-linear oracle: the product with everything near (the dense vertex matrix), the FMM
product, the right-hand side, the energy, the 2 x 2 vertex-block preconditioner and a GMRES
solve; the calls that support only piecewise constants reject the basis. Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, linear  # noqa: E402
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


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def _dev(x):
    return torch.tensor(np.asarray(x), device="cuda", dtype=torch.float64)


def _ctx(m, qr, **kw):
    ctx = pb.pb_create(pb.params(eps_in=1.0, eps_out=80.0, kappa=KAP, qr=qr, basis=pb.PB_BASIS_LINEAR, **kw))
    pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
    pb.pb_build_tree(ctx)
    return ctx


@pytest.fixture(scope="module")
def surf():
    # irregular element sizes (a perturbed sphere), charges inside
    V, T = inputs.perturbed_sphere(3, 3.0, 0.12, seed=31)
    qp, q = inputs.ball_charges(6, 1.8, seed=32)
    return inputs.Mesh(V, T, qp, q)


@pytest.fixture(scope="module")
def dense_p1(surf):
    out = {}
    for qr in (2, 3):
        ph = dense.Phys(1.0, 80.0, KAP, qs=3, qr=qr)
        out[qr] = (ph, linear.assemble(surf, ph))
    return out


@pytest.mark.parametrize("qr", [2, 3, 4])
def test_all_near_equals_dense(surf, qr):
    m = surf
    ph = dense.Phys(1.0, 80.0, KAP, qs=3, qr=qr)
    nv = m.verts.shape[0]
    x = inputs.random_density(nv, 5)
    yo = linear.matvec(m, ph, x)
    for prec, tol in ((pb.PB_FP64, 1e-12), (pb.PB_MIXED, 2e-6)):
        ctx = _ctx(m, qr, leaf_size=16, eta0=1e-6, p=2, precision=prec)
        try:
            y = torch.empty(2 * nv, device="cuda", dtype=torch.float64)
            pb.pb_matvec(ctx, _dev(x), y)
            assert _rel(y.cpu().numpy(), yo) < tol, (qr, prec, _rel(y.cpu().numpy(), yo))
        finally:
            pb.pb_destroy(ctx)


@pytest.mark.parametrize("prec,p,tol", [(pb.PB_FP64, 10, 2e-6), (pb.PB_MIXED, 8, 5e-5)])
def test_fmm_product_within_truncation_of_dense(surf, dense_p1, prec, p, tol):
    m = surf
    ph, A = dense_p1[2]
    nv = m.verts.shape[0]
    x = inputs.random_density(nv, 6)
    ctx = _ctx(m, 2, leaf_size=16, eta0=0.8, p=p, precision=prec)
    try:
        st = pb.pb_get_tree_stats(ctx)
        assert sum(st["ninter"]) > 0  # the far field is in use
        y = torch.empty(2 * nv, device="cuda", dtype=torch.float64)
        pb.pb_matvec(ctx, _dev(x), y)
        assert _rel(y.cpu().numpy(), A @ x) < tol
    finally:
        pb.pb_destroy(ctx)


def test_rhs_energy_and_preconditioner(surf, dense_p1):
    m = surf
    ph, A = dense_p1[3]
    nv = m.verts.shape[0]
    bo = linear.rhs(m, ph)
    xo = np.linalg.solve(A, bo)
    Eo = linear.energy(m, ph, xo)
    # the 2 x 2 diagonal blocks of the vertex system, inverted
    r = inputs.random_density(nv, 7)
    zo = np.empty(2 * nv)
    for v in range(nv):
        D = np.array([[A[v, v], A[v, nv + v]], [A[nv + v, v], A[nv + v, nv + v]]])
        zo[[v, nv + v]] = np.linalg.solve(D, r[[v, nv + v]])
    for prec, tol in ((pb.PB_FP64, 1e-12), (pb.PB_MIXED, 1e-6)):
        ctx = _ctx(m, 3, leaf_size=16, eta0=0.8, p=6, precision=prec)
        try:
            b = torch.empty(2 * nv, device="cuda", dtype=torch.float64)
            pb.pb_rhs(ctx, b)
            assert _rel(b.cpu().numpy(), bo) < tol
            E = pb.pb_solvation_energy(ctx, _dev(xo))
            assert abs(E - Eo) < tol * abs(Eo)
            z = torch.empty(2 * nv, device="cuda", dtype=torch.float64)
            pb.pb_precond_apply(ctx, _dev(r), z)
            assert _rel(z.cpu().numpy(), zo) < 1e-11  # exact FP64 entries in both precisions
        finally:
            pb.pb_destroy(ctx)


@pytest.mark.parametrize("prec", [pb.PB_FP64, pb.PB_MIXED])
def test_gmres_solution_and_energy(surf, dense_p1, prec):
    m = surf
    ph, A = dense_p1[2]
    nv = m.verts.shape[0]
    bo = linear.rhs(m, ph)
    xo = np.linalg.solve(A, bo)
    Eo = linear.energy(m, ph, xo)
    ctx = _ctx(m, 2, leaf_size=16, eta0=0.8, p=10 if prec == pb.PB_FP64 else 8, precision=prec)
    try:
        x = torch.zeros(2 * nv, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-8 if prec == pb.PB_FP64 else 1e-6, max_iter=200, restart=60)
        assert info.status == pb.PB_OK
        E = pb.pb_solvation_energy(ctx, x)
        # the FMM truncation (p) and the solver tolerance are the budget
        assert abs(E - Eo) < (2e-6 if prec == pb.PB_FP64 else 5e-5) * abs(Eo), (E, Eo)
        assert _rel(x.cpu().numpy(), xo) < (1e-5 if prec == pb.PB_FP64 else 2e-4)
    finally:
        pb.pb_destroy(ctx)


def test_kirkwood_sphere_matches_oracle_and_closed_form():
    from oracle import kirkwood

    V, T = inputs.icosphere(3, 2.0)
    m = inputs.Mesh(V, T, np.zeros((1, 3)), np.array([1.0]))
    ph = dense.Phys(1.0, 80.0, KAP, qs=3, qr=2)
    xo, _, _ = linear.solve(m, ph)
    Eo = linear.energy(m, ph, xo)
    ctx = _ctx(m, 2, leaf_size=16, eta0=0.8, p=10, precision=pb.PB_FP64)
    try:
        x = torch.zeros(2 * V.shape[0], device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-10, max_iter=100, restart=50)
        assert info.status == pb.PB_OK
        E = pb.pb_solvation_energy(ctx, x)
        assert abs(E - Eo) < 1e-6 * abs(Eo)
        ref = kirkwood.centered(1.0, 2.0, 1.0, 80.0, KAP)
        assert abs(E - ref) < 0.02 * abs(ref)
    finally:
        pb.pb_destroy(ctx)


def test_piecewise_constant_only_calls_reject_the_basis(surf):
    m = surf
    with pytest.raises(pb.PBError):
        pb.pb_create(pb.params(qr=1, basis=pb.PB_BASIS_LINEAR))  # the points carry the hat functions
    ctx = _ctx(m, 2, leaf_size=16, eta0=0.8, p=4, precision=pb.PB_MIXED)
    nv = m.verts.shape[0]
    try:
        x = _dev(inputs.random_density(nv, 8))
        for call in (lambda: pb.pb_solvation_energy_treecode(ctx, x, 0.5),
                     lambda: pb.pb_matvec_multi(ctx, torch.stack([x, x]), torch.empty((2, 2 * nv), device="cuda",
                                                                                    dtype=torch.float64))):
            with pytest.raises(pb.PBError) as e:
                call()
            assert e.value.code == pb.PB_ERR_ARG
    finally:
        pb.pb_destroy(ctx)
