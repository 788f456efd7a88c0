"""Pins of the Kirkwood reference and of the oracle's solve against it (Section 3.1). CPU only."""
import os

import numpy as np
import pytest

from oracle import dense, kirkwood
from paper_2110_13778_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "kirkwood_table1.txt")


def test_centered_closed_form_values():
    # Table 1 exact energy: a = 50, q = 50, eps2/eps1 = 40, kappa = 0.1257 (inferred)
    assert abs(kirkwood.centered(50.0, 50.0, 1.0, 40.0, 0.1257) - (-8273.31)) < 0.02
    # the 2 A, +1 e sphere of the small Kirkwood workload
    assert abs(kirkwood.centered(1.0, 2.0, 1.0, 80.0, 0.1257) - (-82.1886)) < 1e-3


def test_series_reduces_to_closed_form_and_born_kirkwood():
    for kap in (0.0, 0.1257, 1.0):
        e1 = kirkwood.series([[0, 0, 0]], [1.3], 7.0, 2.0, 60.0, kap)
        e2 = kirkwood.centered(1.3, 7.0, 2.0, 60.0, kap)
        assert abs(e1 - e2) < 1e-12 * abs(e2)
    # kappa = 0: g_n = -(n+1) eps2 gives the Born-Kirkwood multipole factor
    g = kirkwood._g(6, 0.0, 80.0)
    n = np.arange(7)
    fac = (1.0 * (n + 1) + g) / (1.0 * n - g)
    bk = (n + 1) * (1.0 - 80.0) / (1.0 * (n * 1.0 + (n + 1) * 80.0))
    assert np.allclose(fac, bk, rtol=1e-14)
    # the small-kappa limit of the ratio recurrence approaches kappa = 0
    assert np.allclose(kirkwood._g(6, 1e-9, 80.0), g, rtol=1e-6)


@pytest.fixture(scope="module")
def kirk_solutions():
    out = {}
    ph = dense.Phys(1.0, 40.0, 0.1257, qs=3)
    for lev in (2, 3):
        m = inputs.kirkwood_centered(lev, 50.0, 50.0)
        x, A, b = dense.solve(m, ph)
        out[m.nt] = (m, x, dense.energy(m, ph, x))
    return out


def test_oracle_solve_converges_to_kirkwood(kirk_solutions):
    ex = kirkwood.centered(50.0, 50.0, 1.0, 40.0, 0.1257)
    err = {n: abs(v[2] - ex) / abs(ex) for n, v in kirk_solutions.items()}
    assert err[320] < 0.035 and err[1280] < 0.01
    assert err[320] / err[1280] > 2.0  # at least O(N^-1/2) per refinement


def test_oracle_tracks_table1(kirk_solutions):
    rows = np.loadtxt(GOLDEN)
    ex = -8273.31
    for N, E_paper, _ in rows:
        if int(N) in kirk_solutions:
            E = kirk_solutions[int(N)][2]
            tol = {320: 0.015, 1280: 0.0025}[int(N)]
            assert abs(E - E_paper) / abs(ex) < tol, (N, E, E_paper)


def test_oracle_surface_fields(kirk_solutions):
    m, x, _ = kirk_solutions[1280]
    phi, dphi = kirkwood.surface_fields_centered(50.0, 50.0, 1.0, 40.0, 0.1257)
    assert abs(x[m.nt:].mean() / dphi - 1) < 0.015
    assert abs(x[: m.nt].mean() / phi - 1) < 0.05


def test_oracle_offcentre_charges_against_series():
    m = inputs.kirkwood_ball(3, 20.0, 10, 12.0, seed=11)
    ph = dense.Phys(1.0, 80.0, 0.1257, qs=3)
    x, _, _ = dense.solve(m, ph)
    E = dense.energy(m, ph, x)
    ref = kirkwood.series(m.qpos, m.q, 20.0, 1.0, 80.0, 0.1257)
    assert abs(E - ref) < 0.02 * abs(ref)
