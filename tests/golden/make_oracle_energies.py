"""Write tests/golden/oracle_energies.json: solvation energies of the larger synthetic
workloads computed by the CPU oracle alone (dense Galerkin system of Section 2.3, energy of
eqsolengdis), for the GPU energy tests.

Only ``oracle`` and the seeded input generators are called. Workloads:
  * kirkwood_l5 -- Kirkwood sphere with off-centre charges: radius 20 A, icosphere level 5
    (20480 triangles), 50 charges uniform in the ball of radius 16 A, values U[-1, 1] e,
    seed 2000; solved by dense LU (partial pivoting) and, as a cross-check, by the
    matrix-free GMRES;
  * kirkwood_l6 -- the same at level 6 (81920 triangles): matrix-free GMRES to 1e-12;
  * molecule_200 -- a 200-atom protein-like molecule (self-avoiding walk, Gaussian
    isosurface on a 0.9 A grid, seed 3200; ~20k triangles): matrix-free GMRES to 1e-12.
eps_in = 1, eps_out = 80, kappa = 0.1257 / A, singular quadrature qs = 3 throughout.

  python tests/golden/make_oracle_energies.py [name ...]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import dense  # noqa: E402
from paper_2110_13778_gb300 import inputs, molecules  # noqa: E402

OUT = os.path.join(HERE, "oracle_energies.json")
PH = dict(eps1=1.0, eps2=80.0, kappa=0.1257, qs=3)


def workload(name):
    if name == "kirkwood_l5":
        return inputs.kirkwood_ball(5, 20.0, 50, 16.0, 2000)
    if name == "kirkwood_l6":
        return inputs.kirkwood_ball(6, 20.0, 50, 16.0, 2000)
    if name == "molecule_200":
        return molecules.molecule(200, 3200, 0.9)[0]
    raise KeyError(name)


def run(name):
    m = workload(name)
    ph = dense.Phys(**PH)
    rec = {"workload": name, "N": int(m.nt), "nc": int(m.nc), "phys": PH,
           "source": "oracle (dense Galerkin entries, Section 2.3; energy eqsolengdis)"}
    t0 = time.time()
    if name == "kirkwood_l5":
        x, _, _ = dense.solve(m, ph)
        rec["energy_kcal"] = dense.energy(m, ph, x)
        rec["method"] = "dense LU"
        rec["lu_seconds"] = time.time() - t0
        t1 = time.time()
        xg, _, res, nmv = dense.solve_matrix_free(m, ph)
        rec["gmres_energy_kcal"] = dense.energy(m, ph, xg)
        rec["gmres_residual"], rec["gmres_products"], rec["gmres_seconds"] = res, nmv, time.time() - t1
    else:
        x, _, res, nmv = dense.solve_matrix_free(m, ph)
        rec["energy_kcal"] = dense.energy(m, ph, x)
        rec["method"] = "matrix-free GMRES right-scaled by the diagonal mass terms"
        rec["residual"], rec["products"] = res, nmv
        rec["seconds"] = time.time() - t0
    return rec


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names:
        rec = run(name)
        print(json.dumps(rec), flush=True)
        data[name] = rec
        with open(OUT + ".tmp", "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)


if __name__ == "__main__":
    main(sys.argv[1:] or ["kirkwood_l5", "molecule_200", "kirkwood_l6"])
