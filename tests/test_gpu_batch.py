"""Several molecules x several charge states in one CUDA-graph launch (pb_batch_solve_states)
against the same molecules solved one by one (pb_solve_states, batched states) and, for the
small sphere, against the oracle's dense LU energies of every state. Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense  # noqa: E402
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


def _states(m, R, seed):
    rng = np.random.default_rng(seed)
    Q = np.repeat(m.q[None, :], R, axis=0)
    for s in range(1, R):
        flip = rng.random(m.nc) < 0.2
        Q[s, flip] = -Q[s, flip]
    return Q


def _ctx(m, precision):
    ctx = pb.pb_create(pb.params(eps_in=1.0, eps_out=80.0, kappa=KAP, eta0=0.7, leaf_size=32, p=6,
                                 precision=precision, precond=pb.PB_PRECOND_BLOCK))
    pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
    pb.pb_build_tree(ctx)
    return ctx


def _run(mols, R, precision, tol=1e-6):
    # FP64 runs are reproducible to rounding, so the batch must give exactly the one-by-one
    # results; mixed runs sum FP32 partials through atomics and agree to FP32 rounding
    exact = precision == pb.PB_FP64
    Qs = [_states(m, R, 10 + k) for k, m in enumerate(mols)]
    ctxs = [_ctx(m, precision) for m in mols]
    try:
        Xb = [torch.empty((R, 2 * m.nt), device="cuda", dtype=torch.float64) for m in mols]
        g0 = [pb.pb_get_graph_launches(c) for c in ctxs]
        Eb, ib = pb.pb_batch_solve_states(ctxs, Qs, Xb, tol=tol, max_iter=300, restart=40)
        assert [pb.pb_get_graph_launches(c) - g for c, g in zip(ctxs, g0)] == [1] * len(mols)
        for k, (c, m) in enumerate(zip(ctxs, mols)):
            Xr = torch.empty_like(Xb[k])
            Er, ir = pb.pb_solve_states(c, Qs[k], Xr, tol=tol, max_iter=300, restart=40, warm=2)
            for a, b in zip(ib[k], ir):
                assert a.status == b.status == pb.PB_OK
                if exact:
                    assert a.iterations == b.iterations and a.matvecs == b.matvecs
                    assert abs(a.rel_residual - b.rel_residual) <= 1e-6 * b.rel_residual + 1e-15
                else:
                    assert abs(a.iterations - b.iterations) <= 1
                    assert a.rel_residual < 2 * tol and b.rel_residual < 2 * tol
            assert np.allclose(Eb[k], Er, rtol=1e-10 if exact else 1e-6, atol=0)
            assert (Xb[k] - Xr).norm().item() <= (1e-9 if exact else 1e-5) * Xr.norm().item()
        return Eb, Qs
    finally:
        for c in ctxs:
            pb.pb_destroy(c)


@pytest.mark.parametrize("precision", [pb.PB_FP64, pb.PB_MIXED])
def test_three_molecules_five_states(precision):
    sphere = inputs.kirkwood_ball(3, 2.0, 6, 1.5, seed=3)
    mols = [sphere, molecules.molecule(40, 4040, 1.0)[0], molecules.molecule(25, 4025, 1.1)[0]]
    Eb, Qs = _run(mols, 5, precision)
    # the sphere's states against the oracle (dense LU per state)
    ph = dense.Phys(1.0, 80.0, KAP, qs=3)
    A = dense.assemble(sphere.verts, sphere.tris, ph)
    for s in range(5):
        ms = inputs.Mesh(sphere.verts, sphere.tris, sphere.qpos, Qs[0][s])
        x = np.linalg.solve(A, dense.rhs(ms, ph))
        Eo = dense.energy(ms, ph, x)
        assert abs(Eb[0][s] - Eo) < 1e-3 * abs(Eo), (s, Eb[0][s], Eo)


def test_one_state_and_two_batches_of_states():
    m1 = inputs.kirkwood_ball(2, 2.0, 5, 1.5, seed=4)
    m2 = molecules.molecule(20, 4020, 1.2)[0]
    _run([m1, m2], 1, pb.PB_FP64)
    _run([m1, m2], 70, pb.PB_FP64)  # states 1..64 and 65..69 in two batches
