"""Regular quadrature of orders 2-4 (Section 3.1, Table 2) on the GPU against the oracle at
the same order: the product with everything near (the dense Galerkin matrix), the FMM product,
the right-hand side, the energy (direct and treecode) and a solve on the paper's Kirkwood
sphere that lands on Table 2's order-4 energy. Needs a GPU."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, fmm  # noqa: E402
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
    ctx = pb.pb_create(pb.params(eps_in=1.0, eps_out=kw.pop("eps_out", 80.0), kappa=KAP, qr=qr, **kw))
    pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
    pb.pb_build_tree(ctx)
    return ctx


@pytest.fixture(scope="module")
def sphere():
    return inputs.kirkwood_ball(3, 2.0, 5, 1.5, seed=3)


@pytest.mark.parametrize("qr", [2, 3, 4])
def test_all_near_equals_dense(sphere, qr):
    m = sphere
    ph = dense.Phys(1.0, 80.0, KAP, qs=3, qr=qr)
    A = dense.assemble(m.verts, m.tris, ph)
    for prec, tol in ((pb.PB_FP64, 1e-12), (pb.PB_MIXED, 2e-6)):
        ctx = _ctx(m, qr, leaf_size=16, eta0=1e-6, p=2, precision=prec, singular=pb.PB_SINGULAR_FP64)
        try:
            x = inputs.random_density(m.nt, 5)
            y = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
            pb.pb_matvec(ctx, _dev(x), y)
            assert _rel(y.cpu().numpy(), A @ x) < tol, (qr, prec)
        finally:
            pb.pb_destroy(ctx)


@pytest.mark.parametrize("qr,prec", [(2, pb.PB_FP64), (3, pb.PB_FP64), (2, pb.PB_MIXED)])
def test_fmm_matches_oracle_fmm(sphere, qr, prec):
    m = sphere
    ph = dense.Phys(1.0, 80.0, KAP, qs=3, qr=qr)
    A = dense.assemble(m.verts, m.tris, ph)
    ctx = _ctx(m, qr, leaf_size=16, eta0=0.8, p=6, precision=prec)
    try:
        x = inputs.random_density(m.nt, 9)
        y = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
        pb.pb_matvec(ctx, _dev(x), y)
        tr = fmm.Tree(m.verts, m.tris, leaf_size=16, eta0=0.8)
        yo = fmm.matvec(tr, m.verts, m.tris, x, ph, 6, A=A)
        assert _rel(y.cpu().numpy(), yo) < (1e-10 if prec == pb.PB_FP64 else 2e-5)
        # several vectors at once (one at a time inside) give the same products
        X = torch.stack([_dev(x), _dev(2 * x)])
        Y = torch.empty_like(X)
        pb.pb_matvec_multi(ctx, X, Y)
        assert _rel(Y[1].cpu().numpy(), 2 * yo) < (1e-10 if prec == pb.PB_FP64 else 2e-5)
    finally:
        pb.pb_destroy(ctx)


@pytest.mark.parametrize("qr", [2, 4])
def test_rhs_energy_and_treecode(sphere, qr):
    m = sphere
    ph = dense.Phys(1.0, 80.0, KAP, qs=3, qr=qr)
    A = dense.assemble(m.verts, m.tris, ph)
    bo = dense.rhs(m, ph)
    xo = np.linalg.solve(A, bo)
    for prec, tol in ((pb.PB_FP64, 1e-12), (pb.PB_MIXED, 1e-6)):
        ctx = _ctx(m, qr, leaf_size=16, eta0=0.8, p=6, precision=prec)
        try:
            b = torch.empty(2 * m.nt, device="cuda", dtype=torch.float64)
            pb.pb_rhs(ctx, b)
            assert _rel(b.cpu().numpy(), bo) < tol
            E = pb.pb_solvation_energy(ctx, _dev(xo))
            Eo = dense.energy(m, ph, xo)
            assert abs(E - Eo) < tol * abs(Eo)
            if prec == pb.PB_FP64:
                tr = fmm.Tree(m.verts, m.tris, leaf_size=16, eta0=0.8)
                Et = pb.pb_solvation_energy_treecode(ctx, _dev(xo), 0.5)
                Eto = fmm.treecode_energy(tr, m, xo, ph, 6, 0.5)
                assert abs(Et - Eto) < 1e-10 * abs(Eto)
        finally:
            pb.pb_destroy(ctx)


def test_table2_order4_solve():
    # the paper's sphere (radius 50 A, 50 e at the centre, eps 1/40) at N = 320 with the
    # order-4 rule: the oracle's dense solve, and Table 2's value within the oracle's own bar
    m = inputs.kirkwood_centered(2, 50.0, 50.0)
    ph = dense.Phys(1.0, 40.0, KAP, qs=3, qr=4)
    xo, _, _ = dense.solve(m, ph)
    Eo = dense.energy(m, ph, xo)
    rows = {int(r[0]): r[1:] for r in np.loadtxt(os.path.join(os.path.dirname(__file__), "golden",
                                                               "kirkwood_table2.txt"))}
    ctx = _ctx(m, 4, leaf_size=16, eta0=0.8, p=8, precision=pb.PB_FP64, eps_out=40.0)
    try:
        x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-10, max_iter=100, restart=50)
        assert info.status == pb.PB_OK
        E = pb.pb_solvation_energy(ctx, x)
        assert abs(E - Eo) < 1e-6 * abs(Eo)
        assert abs(E - rows[320][2]) / 8273.31 < 3e-4
    finally:
        pb.pb_destroy(ctx)


def test_batched_states_need_order_one(sphere):
    ctx = _ctx(sphere, 2, leaf_size=16, eta0=0.8, p=4, precision=pb.PB_MIXED)
    try:
        Q = np.repeat(sphere.q[None, :], 3, axis=0)
        X = torch.empty((3, 2 * sphere.nt), device="cuda", dtype=torch.float64)
        with pytest.raises(pb.PBError) as e:
            pb.pb_solve_states(ctx, Q, X, warm=2)
        assert e.value.code == pb.PB_ERR_ARG
        E, infos = pb.pb_solve_states(ctx, Q, X, warm=1)  # one at a time is fine
        assert all(i.status == pb.PB_OK for i in infos)
    finally:
        pb.pb_destroy(ctx)
