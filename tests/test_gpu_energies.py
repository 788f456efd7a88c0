"""Solvation energies of the larger workloads against the oracle: the Kirkwood sphere with
off-centre charges at icosphere levels 5 and 6 (20480 and 81920 triangles) and a 200-atom
protein-like molecule (~20k triangles), each against the oracle's energy stored in
tests/golden/oracle_energies.json (written by tests/golden/make_oracle_energies.py, which
calls only the oracle). Both precisions, FMM order 8, the benchmark's settings (leaf 64,
eta0 0.8, block-diagonal preconditioner, GMRES to 1e-6). Bar: 1e-3 relative. Needs a GPU."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2110_13778_gb300 import inputs, molecules, pb  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_energies.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_13778_gb300 import build

    build.build()
    pb.lib()


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _workload(name):
    # the same seeded inputs the golden script used
    if name == "kirkwood_l5":
        return inputs.kirkwood_ball(5, 20.0, 50, 16.0, 2000)
    if name == "kirkwood_l6":
        return inputs.kirkwood_ball(6, 20.0, 50, 16.0, 2000)
    return molecules.molecule(200, 3200, 0.9)[0]


@pytest.mark.parametrize("name", ["kirkwood_l5", "molecule_200", "kirkwood_l6"])
@pytest.mark.parametrize("precision", [pb.PB_MIXED, pb.PB_FP64])
def test_energy_matches_oracle(name, precision):
    g = _golden()[name]
    m = _workload(name)
    assert m.nt == g["N"] and m.nc == g["nc"]
    ph = g["phys"]
    ctx = pb.pb_create(pb.params(eps_in=ph["eps1"], eps_out=ph["eps2"], kappa=ph["kappa"], eta0=0.8, leaf_size=64,
                                 p=8, qs=ph["qs"], precision=precision, precond=pb.PB_PRECOND_BLOCK))
    try:
        pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
        pb.pb_build_tree(ctx)
        x = torch.zeros(2 * m.nt, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=500, restart=50)
        assert info.status == pb.PB_OK
        E = pb.pb_solvation_energy(ctx, x)
        Eo = g["energy_kcal"]
        err = abs(E - Eo) / abs(Eo)
        print(f"{name} precision {precision}: E {E:.8f} oracle {Eo:.8f} rel {err:.2e} iters {info.iterations}")
        assert np.isfinite(E) and err < 1e-3
    finally:
        pb.pb_destroy(ctx)
