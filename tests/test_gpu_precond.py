"""Diagonal ("d") against block-diagonal ("bd") preconditioning (Section 2.6, Table 4) on a
protein-like surface whose marching-tetrahedra triangulation has the narrow and tiny
triangles the paper blames for ill-conditioning, and the block size that stands for the
designated level. Every preconditioner must give the same solution; bd must need fewer
iterations than d and than no preconditioner. Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2110_13778_gb300 import molecules, pb  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_13778_gb300 import build

    build.build()
    pb.lib()


def _solve(m, precond, pc_block=0):
    ctx = pb.pb_create(pb.params(eps_in=1.0, eps_out=80.0, kappa=0.1257, eta0=0.8, leaf_size=64, p=8,
                                 precision=pb.PB_MIXED, precond=precond, pc_block=pc_block))
    try:
        pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
        pb.pb_build_tree(ctx)
        x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=600, restart=50, raise_on_fail=False)
        st = pb.pb_get_tree_stats(ctx)
        return x, info, pb.pb_solvation_energy(ctx, x), st
    finally:
        pb.pb_destroy(ctx)


def test_block_diagonal_beats_diagonal_and_all_agree():
    m = molecules.molecule(150, 3150, 0.9)[0]
    # the triangulation has slivers: the smallest element is far below the mean
    from oracle import dense

    _, area, _ = dense.geometry(m.verts, m.tris)
    assert area.min() < 1e-2 * area.mean()
    runs = {"none": _solve(m, pb.PB_PRECOND_NONE), "d": _solve(m, pb.PB_PRECOND_DIAG)}
    for b in (16, 32, 64, 96):
        runs[f"bd{b}"] = _solve(m, pb.PB_PRECOND_BLOCK, b)
    its = {k: v[1].iterations for k, v in runs.items()}
    ok = {k: v[1].status == pb.PB_OK for k, v in runs.items()}
    print(its, ok)
    # every block form converges; without a preconditioner (or with the 2 x 2 diagonal) the
    # slivers may stall restarted GMRES altogether: then it has used its whole budget
    for b in (16, 32, 64, 96):
        assert ok[f"bd{b}"], b
    for k in ("none", "d"):
        assert ok[k] or its[k] == 600
    assert its["bd96"] < its["d"] and its["bd96"] < its["none"]
    assert its["bd96"] <= its["bd16"]
    # smaller blocks: more of them
    assert runs["bd16"][3]["pc_blocks"] > runs["bd96"][3]["pc_blocks"]
    assert runs["bd16"][3]["pc_max"] <= 32
    E0 = runs["bd96"][2]
    x0 = runs["bd96"][0]
    for k, v in runs.items():
        if ok[k]:
            assert abs(v[2] - E0) < 1e-5 * abs(E0), k
            assert (v[0] - x0).norm().item() < 2e-5 * x0.norm().item(), k


def test_pc_block_rejected_out_of_range():
    for b in (4, 97):
        with pytest.raises(pb.PBError):
            pb.pb_create(pb.params(pc_block=b))
