"""Learned warm start on the GPU: the BF16 tensor-core network kernels and the feature kernel
against the FP64 oracle (oracle/mlp.py), and what a trained network gains. Needs a GPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as omlp  # noqa: E402
from paper_2110_13778_gb300 import molecules, pb, warmstart  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPE = (18, 128, 3, 2)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2110_13778_gb300 import build

    build.build()
    pb.lib()


@pytest.fixture
def net():
    h = pb.pb_mlp_create(*SHAPE, seed=5)
    yield h
    pb.pb_mlp_destroy(h)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / np.linalg.norm(b))


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, SHAPE[0])).astype(np.float32)
    T = rng.standard_normal((n, SHAPE[3])).astype(np.float32)
    return X, T


def test_init_and_param_roundtrip(net):
    w = pb.pb_mlp_get_params(net)
    lay, n = omlp.layout(*SHAPE)
    assert w.size == n
    layers = omlp.unpack(w.astype(np.float64), SHAPE)
    assert np.all(layers[0][0][:, 18:] == 0) and np.all(layers[-1][0][2:, :] == 0)
    for l, (W, b) in enumerate(layers):
        assert np.all(b == 0)
        fan = (18 if l == 0 else 128) + (128 if l < 3 else 2)
        assert np.abs(W).max() <= np.sqrt(6.0 / fan) * (1 + 1e-6)
    w2 = omlp.init_params(SHAPE, 9).astype(np.float32)
    pb.pb_mlp_set_params(net, w2)
    np.testing.assert_array_equal(pb.pb_mlp_get_params(net), w2)


@pytest.mark.parametrize("n", [1, 37, 4096 + 77])
def test_forward_matches_oracle(net, n):
    w = omlp.init_params(SHAPE, 1).astype(np.float32)
    pb.pb_mlp_set_params(net, w)
    X, _ = _data(n, n)
    Y = torch.empty((n, 2), device="cuda", dtype=torch.float32)
    pb.pb_mlp_forward(net, torch.from_numpy(X).cuda(), Y)
    y = Y.cpu().numpy()
    ye, _ = omlp.forward(w.astype(np.float64), SHAPE, X.astype(np.float64), emulate=True)
    yf, _ = omlp.forward(w.astype(np.float64), SHAPE, X.astype(np.float64))
    # bfloat16 rounding at the same points: FP32 accumulation order is the only difference
    assert _rel(y, ye) < 2e-3
    # and the bfloat16 error against the exact FP64 network stays at bfloat16's level
    assert _rel(y, yf) < 3e-2


@pytest.mark.parametrize("shape", [(5, 64, 2, 3), (16, 128, 1, 17), (40, 128, 2, 2)])
def test_forward_layered_path_matches_oracle(shape):
    # shapes outside the fused kernel (width != 128, > 16 outputs, > 32 inputs) take the
    # layer-by-layer tensor-core GEMMs
    h = pb.pb_mlp_create(*shape, seed=3)
    try:
        w = omlp.init_params(shape, 4).astype(np.float32)
        pb.pb_mlp_set_params(h, w)
        X = np.random.default_rng(9).standard_normal((300, shape[0])).astype(np.float32)
        Y = torch.empty((300, shape[3]), device="cuda", dtype=torch.float32)
        pb.pb_mlp_forward(h, torch.from_numpy(X).cuda(), Y)
        ye, _ = omlp.forward(w.astype(np.float64), shape, X.astype(np.float64), emulate=True)
        assert _rel(Y.cpu().numpy(), ye) < 2e-3
    finally:
        pb.pb_mlp_destroy(h)


@pytest.mark.parametrize("n", [19, 20000 + 5])
def test_gradient_matches_oracle(net, n):
    w = omlp.init_params(SHAPE, 2).astype(np.float32)
    pb.pb_mlp_set_params(net, w)
    X, T = _data(n, 100 + n)
    loss, g = pb.pb_mlp_gradient(net, torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    lo, go = omlp.loss_grad(w.astype(np.float64), SHAPE, X.astype(np.float64), T.astype(np.float64), emulate=True)
    assert abs(loss - lo) < 1e-3 * lo
    G = omlp.unpack(g.astype(np.float64), SHAPE)
    Go = omlp.unpack(go, SHAPE)
    for (gw, gb), (ow, ob) in zip(G, Go):
        assert _rel(gw, ow) < 2e-2
        assert _rel(gb, ob) < 2e-2
    # padded entries get no gradient
    lay, _ = omlp.layout(*SHAPE)
    assert np.all(G[0][0][:, 18:] == 0) and np.all(G[-1][0][2:, :] == 0) and np.all(G[-1][1][2:] == 0)


def test_adam_step_matches_oracle(net):
    w = omlp.init_params(SHAPE, 3).astype(np.float32)
    pb.pb_mlp_set_params(net, w)
    X, T = _data(3000, 7)
    Xd, Td = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    w64 = w.astype(np.float64)
    m, v = np.zeros_like(w64), np.zeros_like(w64)
    for t in (1, 2, 3):
        _, g = pb.pb_mlp_gradient(net, Xd, Td)
        pb.pb_mlp_train_step(net, Xd, Td, 1e-3)
        omlp.adam_step(w64, m, v, g.astype(np.float64), t, 1e-3)
        wg = pb.pb_mlp_get_params(net).astype(np.float64)
        np.testing.assert_allclose(wg, w64, rtol=0, atol=1e-6)
        w64 = wg.copy()  # follow the GPU's FP32 weights


def test_training_reduces_loss(net):
    rng = np.random.default_rng(8)
    X = rng.uniform(-1, 1, (8192, 18)).astype(np.float32)
    T = np.stack([np.sin(2 * X[:, 0]) * X[:, 1], X[:, 2] ** 2 - X[:, 3]], axis=1).astype(np.float32)
    F, Tt = torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda()
    first, last, _ = warmstart.train(net, F, Tt, steps=600, batch=2048, lr=3e-3, lr_final=3e-4)
    assert last < 0.05 * first


@pytest.fixture(scope="module")
def mol():
    return molecules.molecule(40, 4040, 1.0)[0]


def test_features_match_oracle(mol):
    prm = warmstart.solve_params()
    ctx = pb.pb_create(prm)
    try:
        pb.pb_mesh_upload(ctx, mol.verts, mol.tris, mol.qpos, mol.q)
        pb.pb_build_tree(ctx)
        x = torch.zeros(2 * mol.nt, device="cuda", dtype=torch.float64)
        pb.pb_gmres_solve(ctx, x, tol=1e-6, max_iter=300, restart=50)
        F = torch.empty((mol.nt, 18), device="cuda", dtype=torch.float32)
        T = torch.empty((mol.nt, 2), device="cuda", dtype=torch.float32)
        sc = pb.pb_features(ctx, F, x, T)
        Fo, sco, To = omlp.features(mol, prm.eps_in, x.cpu().numpy(), eps_out=prm.eps_out, kappa=prm.kappa)
        # the charge sums run in FP32 per tile of 256 charges, FP64 across tiles
        np.testing.assert_allclose(sc, sco, rtol=2e-5)
        np.testing.assert_allclose(F.cpu().numpy(), Fo, rtol=1e-4, atol=1e-4)
        np.testing.assert_allclose(T.cpu().numpy(), To, rtol=1e-4, atol=1e-4 * np.abs(To).max())
        # features without targets, and the argument check
        pb.pb_features(ctx, F)
        with pytest.raises(pb.PBError):
            pb.pb_features(ctx, F, x, None)
    finally:
        pb.pb_destroy(ctx)


def test_trained_network_saves_iterations(mol):
    prm = warmstart.solve_params()
    F, T = warmstart.make_dataset([30, 40, 50, 60, 35, 45, 55, 65], seed=77, prm=prm)
    net = pb.pb_mlp_create(*SHAPE, seed=11)
    try:
        first, last, _ = warmstart.train(net, F, T, steps=2000, batch=4096, lr=1e-3, lr_final=1e-4)
        assert last < 0.2 * first
        for pc in (pb.PB_PRECOND_BLOCK, pb.PB_PRECOND_DIAG):
            res = warmstart.evaluate(net, mol, warmstart.solve_params(precond=pc))
            z, l = res["zero"], res["learned"]
            assert z["info"].status == pb.PB_OK and l["info"].status == pb.PB_OK
            # GMRES is the judge: the same energy to the solve tolerance
            assert abs(l["energy"] - z["energy"]) < 1e-4 * abs(z["energy"])
            # the prediction removes most of the initial residual and never costs iterations
            assert z["info"].initial_residual == 1.0
            assert l["info"].initial_residual < 0.4, l["info"].initial_residual
            assert l["info"].iterations <= z["info"].iterations, (l["info"].iterations, z["info"].iterations)
    finally:
        pb.pb_mlp_destroy(net)
