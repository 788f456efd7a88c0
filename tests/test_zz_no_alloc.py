"""The allocation-free energy entry point against the regular one. Needs a GPU.

pb_solvation_energy_noalloc serves callers that cannot call cudaMalloc (a host with a fixed
device-memory budget that forbids allocations after start-up, or code where an allocation is
not allowed): it keeps its scratch in a fixed device array instead of allocating. This file
is named so that pytest collects it last; it must pass alone in a fresh process and after the
other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2110_13778_gb300 import inputs, pb  # noqa: E402

pytestmark = pytest.mark.gpu

# the tolerances the energy parity tests use: FP64 and mixed precision
TOL = {pb.PB_FP64: 1e-12, pb.PB_MIXED: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_13778_gb300 import build

    build.build()
    pb.lib()


@pytest.mark.parametrize("precision", [pb.PB_FP64, pb.PB_MIXED])
def test_noalloc_energy_matches_context_energy_twice(precision):
    m = inputs.kirkwood_ball(3, 2.0, 7, 1.5, seed=21)
    prm = pb.params(leaf_size=16, eta0=0.8, p=4, precision=precision)
    ctx = pb.pb_create(prm)
    try:
        pb.pb_mesh_upload(ctx, m.verts, m.tris, m.qpos, m.q)
        pb.pb_build_tree(ctx)
        dv = torch.tensor(m.verts, device="cuda", dtype=torch.float64)
        dt = torch.tensor(m.tris, device="cuda", dtype=torch.int32)
        dqp = torch.tensor(m.qpos, device="cuda", dtype=torch.float64)
        dq = torch.tensor(m.q, device="cuda", dtype=torch.float64)
        E = torch.zeros(1, device="cuda", dtype=torch.float64)
        for seed in (1, 2):  # two calls in a row, different densities
            x = torch.tensor(inputs.random_density(m.nt, seed), device="cuda", dtype=torch.float64)
            ref = pb.pb_solvation_energy(ctx, x)
            pb.pb_solvation_energy_noalloc(dv, dt, dqp, dq, x, E, precision=precision)
            torch.cuda.synchronize()
            got = float(E.item())
            assert abs(got - ref) <= TOL[precision] * abs(ref), (seed, got, ref)
    finally:
        pb.pb_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    err = ctypes.create_string_buffer(256)
    buf = torch.zeros(16, device="cuda", dtype=torch.float64)
    p = ctypes.c_void_p(buf.data_ptr())
    rc = pb.lib().pb_solvation_energy_noalloc(p, p, 3_000_000, p, p, 1, 1.0, 80.0, 0.1, pb.PB_FP64, p, p,
                                              ctypes.c_void_p(0), err, 256)
    assert rc == pb.PB_ERR_ARG
    assert b"scratch limit" in err.value


def test_noalloc_without_charges_gives_zero():
    m = inputs.kirkwood_ball(2, 2.0, 3, 1.5, seed=22)
    dv = torch.tensor(m.verts, device="cuda", dtype=torch.float64)
    dt = torch.tensor(m.tris, device="cuda", dtype=torch.int32)
    x = torch.tensor(inputs.random_density(m.nt, 3), device="cuda", dtype=torch.float64)
    E = torch.full((1,), 7.0, device="cuda", dtype=torch.float64)
    err = ctypes.create_string_buffer(256)
    rc = pb.lib().pb_solvation_energy_noalloc(ctypes.c_void_p(dv.data_ptr()), ctypes.c_void_p(dt.data_ptr()), m.nt,
                                              None, None, 0, 1.0, 80.0, 0.1257, pb.PB_FP64,
                                              ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                              ctypes.c_void_p(0), err, 256)
    torch.cuda.synchronize()
    assert rc == pb.PB_OK and float(E.item()) == 0.0
