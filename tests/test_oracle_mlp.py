"""Pins of the warm-start oracle (oracle/mlp.py) against facts fixed outside it: finite
differences, closed forms, torch's own bfloat16 rounding and the exact features of a regular
octahedron around a point charge. CPU only."""
import numpy as np
import pytest

from oracle import dense
from oracle import mlp
from paper_2110_13778_gb300.inputs import Mesh, icosphere, ball_charges

torch = pytest.importorskip("torch")


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(20000).astype(np.float32) * np.float32(10.0) ** rng.integers(-20, 20, 20000)
    # exact ties: a bfloat16 value plus half an ulp, both parities
    base = np.arange(1, 200, dtype=np.uint32) << 16
    ties = (base | 0x8000).view(np.float32)
    x = np.concatenate([x, ties, -ties, np.float32([0.0, -0.0, 1e-40, 3.4e38])])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_layout_padding():
    lay, n = mlp.layout(12, 128, 3, 2)
    assert [(a, b) for a, b, _, _ in lay] == [(16, 128), (128, 128), (128, 128), (128, 16)]
    assert n == 16 * 128 + 2 * 128 * 128 + 128 * 16 + 3 * 128 + 16
    lay, n = mlp.layout(17, 32, 1, 3)
    assert [(a, b) for a, b, _, _ in lay] == [(32, 32), (32, 16)]


def test_gradient_matches_finite_differences():
    shape = (5, 16, 2, 3)
    rng = np.random.default_rng(1)
    w = mlp.init_params(shape, 3)
    X = rng.standard_normal((9, 5))
    T = rng.standard_normal((9, 3))
    loss, g = mlp.loss_grad(w, shape, X, T)
    lay, n = mlp.layout(*shape)
    # the real (unpadded) parameters
    real = np.zeros(n, dtype=bool)
    for l, (W, b) in enumerate(mlp.unpack(real, shape)):
        rin = 5 if l == 0 else 16
        rout = 16 if l < 2 else 3
        W[:rout, :rin] = True
        b[:rout] = True
    assert np.all(g[~real] == 0.0)
    idx = rng.choice(np.flatnonzero(real), 80, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_grad(wp, shape, X, T)[0] - mlp.loss_grad(wm, shape, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_forward_closed_form():
    # hidden units: x0, x1, x2, -x0, -x1, -x2 (then ReLU); outputs x0 + 2|x1| and relu(x2) + 0.5
    shape = (3, 16, 1, 2)
    lay, n = mlp.layout(*shape)
    w = np.zeros(n)
    (W0, b0), (W1, b1) = mlp.unpack(w, shape)
    for j in range(3):
        W0[j, j] = 1.0
        W0[3 + j, j] = -1.0
    W1[0, 0], W1[0, 3] = 1.0, -1.0
    W1[0, 1], W1[0, 4] = 2.0, 2.0
    W1[1, 2] = 1.0
    b1[1] = 0.5
    X = np.random.default_rng(2).standard_normal((11, 3))
    y, _ = mlp.forward(w, shape, X)
    np.testing.assert_allclose(y[:, 0], X[:, 0] + 2 * np.abs(X[:, 1]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(y[:, 1], np.maximum(X[:, 2], 0) + 0.5, rtol=0, atol=1e-15)
    # with bfloat16 rounding the same values, each rounded where the tensor cores see it
    ye, _ = mlp.forward(w, shape, X, emulate=True)
    xb = mlp.bf16(X)
    np.testing.assert_allclose(ye[:, 0], xb[:, 0] + 2 * np.abs(xb[:, 1]), rtol=0, atol=1e-15)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    w0 = rng.standard_normal(50)
    g = rng.standard_normal(50) * 10.0 ** rng.integers(-4, 3, 50)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    mlp.adam_step(w, m, v, g, 1, 1e-2)
    np.testing.assert_allclose(w, w0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=1e-16)


def test_training_fits_a_smooth_function():
    shape = (2, 32, 2, 1)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (256, 2))
    T = (np.sin(2 * X[:, 0]) * X[:, 1])[:, None]
    w = mlp.init_params(shape, 5)
    m, v = np.zeros_like(w), np.zeros_like(w)
    l0 = mlp.loss_grad(w, shape, X, T)[0]
    for t in range(1, 601):
        loss, g = mlp.loss_grad(w, shape, X, T)
        mlp.adam_step(w, m, v, g, t, 1e-2)
    assert loss < 0.05 * l0


def _octahedron(R):
    V = np.array([[R, 0, 0], [-R, 0, 0], [0, R, 0], [0, -R, 0], [0, 0, R], [0, 0, -R]], float)
    T = []
    for sx, ix in ((1, 0), (-1, 1)):
        for sy, iy in ((1, 2), (-1, 3)):
            for sz, iz in ((1, 4), (-1, 5)):
                t = [ix, iy, iz]
                if sx * sy * sz < 0:
                    t = [ix, iz, iy]
                T.append(t)
    return V, np.array(T, np.int32)


def test_features_of_octahedron_closed_form():
    R, q, eps, eps_out, kap = 3.0, 0.7, 2.0, 80.0, 0.2
    V, T = _octahedron(R)
    m = Mesh(V, T, np.zeros((1, 3)), np.array([q]))
    x = np.arange(16.0)
    F, sc, Tg = mlp.features(m, eps, x, eps_out=eps_out, kappa=kap)
    assert F.shape == (8, 18) and sc.shape == (20,)
    s3 = np.sqrt(3.0)
    c = np.sign(F[:, 0:3])  # (+-1, +-1, +-1): the face's octant
    np.testing.assert_allclose(F[:, 0:3], c / s3, atol=1e-14)  # centroid R c / 3 over R / sqrt 3
    np.testing.assert_allclose(F[:, 3:6], c / s3, atol=1e-14)  # outward normal
    np.testing.assert_allclose(F[:, 6], 0.0, atol=1e-14)
    np.testing.assert_allclose(F[:, 7], 1.0, atol=1e-14)  # mean normal product over 6 neighbours is 0
    np.testing.assert_allclose(F[:, 8], 1.0, atol=1e-14)
    np.testing.assert_allclose(F[:, 9], -1.0, atol=1e-14)
    np.testing.assert_allclose(F[:, 10], 1.0, atol=1e-14)
    np.testing.assert_allclose(F[:, 11], R / (3 * s3), atol=1e-14)
    np.testing.assert_allclose(F[:, 12:15], 1.0, atol=1e-14)  # constant sources over their rms
    np.testing.assert_allclose(F[:, 15], np.exp(-R * R / 150.0) / 10.0, rtol=1e-14)  # r^2 = R^2 / 3
    np.testing.assert_allclose(F[:, 16:18], -1.0, atol=1e-14)  # n . (c - 0) = r > 0
    rc = R / s3  # centroid distance
    np.testing.assert_allclose(sc[8], q / (4 * np.pi * eps * rc), rtol=1e-14)
    np.testing.assert_allclose(sc[9], q / (4 * np.pi * eps * rc * rc), rtol=1e-14)
    np.testing.assert_allclose(sc[12], q * np.exp(-kap * rc) / (4 * np.pi * eps * rc), rtol=1e-14)
    np.testing.assert_allclose(sc[13], q / (4 * np.pi * eps * np.sqrt(rc * rc + 16)), rtol=1e-14)
    np.testing.assert_allclose(sc[14], q / (4 * np.pi * eps * np.sqrt(rc * rc + 64)), rtol=1e-14)
    np.testing.assert_allclose(sc[16], q * rc / (4 * np.pi * eps * (rc * rc + 16) ** 1.5), rtol=1e-14)
    np.testing.assert_allclose(sc[17], q * rc / (4 * np.pi * eps * (rc * rc + 64) ** 1.5), rtol=1e-14)
    np.testing.assert_allclose(sc[6], s3 / 2 * R * R, rtol=1e-14)
    np.testing.assert_allclose(sc[18], sc[8] * 2 * eps / (eps + eps_out), rtol=1e-14)
    np.testing.assert_allclose(sc[19], sc[9] * 2 * eps_out / (eps + eps_out), rtol=1e-14)
    np.testing.assert_allclose(Tg[:, 0], x[:8] / sc[18], rtol=1e-14)
    np.testing.assert_allclose(Tg[:, 1], x[8:] / sc[19], rtol=1e-14)


def test_source_features_match_the_oracle_rhs():
    # S1, S2 at the centroid times the area are the one-point right-hand side (C oracle)
    V, T = icosphere(2, 5.0)
    qp, q = ball_charges(6, 3.0, 11)
    m = Mesh(V, T, qp, q)
    eps = 2.0
    F, sc, _ = mlp.features(m, eps)
    b = dense.rhs(m, dense.Phys(eps, 80.0, 0.1, qs=3))
    A = 0.5 * np.linalg.norm(np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]), axis=1)
    np.testing.assert_allclose(F[:, 8] * sc[8] * A, b[: m.nt], rtol=1e-12)
    np.testing.assert_allclose(F[:, 9] * sc[9] * A, b[m.nt:], rtol=1e-12)


def test_features_invariances():
    V, T = icosphere(2, 5.0)
    qp, q = ball_charges(4, 3.0, 12)
    F, sc, _ = mlp.features(Mesh(V, T, qp, q), 1.0)
    shift = np.array([3.0, -7.0, 11.0])
    Fs, _, _ = mlp.features(Mesh(V + shift, T, qp + shift, q), 1.0)
    np.testing.assert_allclose(Fs, F, atol=1e-12)
    Fk, _, _ = mlp.features(Mesh(2.0 * V, T, 2.0 * qp, q), 1.0)
    np.testing.assert_allclose(Fk[:, :11], F[:, :11], atol=1e-12)  # scale-free columns
    np.testing.assert_allclose(Fk[:, 11], 2.0 * F[:, 11], rtol=1e-12)
    # with kappa = 0 the screened source is S1 itself
    F0, _, _ = mlp.features(Mesh(V, T, qp, q), 1.0, kappa=0.0)
    np.testing.assert_allclose(F0[:, 12], F0[:, 8], rtol=1e-12)
    # smoothing keeps the sources close to S1 and S2
    assert np.corrcoef(F[:, 13], F[:, 8])[0, 1] > 0.9 and np.corrcoef(F[:, 16], F[:, 9])[0, 1] > 0.9
