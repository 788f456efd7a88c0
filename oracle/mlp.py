"""The learned warm start's network and features, in plain FP64 numpy.

TEST INFRASTRUCTURE. This is the oracle for the BF16 tensor-core network kernels and the
feature kernel of the CUDA path. The paper starts GMRES from zero (Section 2.6); the warm
start is an addition, so there is no printed algorithm to follow -- each function below is
the textbook definition written out:

  * Network: layer l computes z_l = W_l a_l + b_l, a_{l+1} = max(z_l, 0) for hidden layers
    and the output is z_L (linear). Parameters are held in the padded layout of the C ABI:
    every W_l (rows = outputs, columns = inputs, row-major) in order, then every b_l; the
    first layer's inputs and the last layer's outputs are padded to multiples of 16.
  * Loss: mean over rows and real outputs of (y - t)^2.
  * Backward pass: reverse-mode differentiation of the two lines above (dz_L = 2 (y - t) /
    (n nout); dW_l = dz_l^T a_l; db_l = column sums of dz_l; da_l = dz_l W_l;
    dz_{l-1} = da_l * [z_{l-1} > 0]).
  * Adam (Kingma and Ba, 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
    w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
  * ``emulate=True`` rounds to bfloat16 (round to nearest, ties to even, on the FP32 value)
    exactly where the CUDA path stores BF16: the weights fed to the tensor cores, the input
    and hidden activations, and the output-layer and back-propagated errors. Everything
    else stays FP64, so the only differences left against the GPU are FP32 accumulation
    order and rare rounding-boundary flips.

Pins (tests/test_oracle_mlp.py): central finite differences of the FP64 loss against the
backward pass; a hand-built network whose output is a known closed form (non-square layers,
so a transposed operand fails); Adam's first step, which is -lr g / (|g| + eps); bfloat16
rounding against torch's own float32 -> bfloat16 conversion; the features of a regular
octahedron around a central charge, where every column is known in closed form; S1 and S2
times the area against the C oracle's right-hand side; invariance under translation and
scaling.
"""
from __future__ import annotations

import numpy as np

NFEAT = 18
NSTAT = 20


def _pad16(x: int) -> int:
    return (x + 15) // 16 * 16


def layout(nin: int, width: int, depth: int, nout: int):
    """[(din, dout, woff, boff) per layer], nparam in the padded C layout."""
    dims = []
    for l in range(depth + 1):
        din = _pad16(nin) if l == 0 else width
        dout = width if l < depth else _pad16(nout)
        dims.append((din, dout))
    out, off = [], 0
    woffs = []
    for din, dout in dims:
        woffs.append(off)
        off += din * dout
    boffs = []
    for din, dout in dims:
        boffs.append(off)
        off += dout
    for (din, dout), wo, bo in zip(dims, woffs, boffs):
        out.append((din, dout, wo, bo))
    return out, off


def unpack(w, shape):
    """Views (W_l, b_l) of the flat parameter vector w for shape = (nin, width, depth, nout)."""
    lay, n = layout(*shape)
    assert w.size == n
    return [(w[wo:wo + din * dout].reshape(dout, din), w[bo:bo + dout]) for din, dout, wo, bo in lay]


def bf16(x):
    """Round to the nearest bfloat16 (ties to even) of the float32 value; returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    out = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def _r(x, emulate):
    return bf16(x) if emulate else x


def forward(w, shape, X, emulate=False):
    """Network output (n x nout) and the per-layer (a_l, z_l) the backward pass needs."""
    nin, width, depth, nout = shape
    layers = unpack(np.asarray(w, dtype=np.float64), shape)
    n = X.shape[0]
    a = np.zeros((n, layers[0][0].shape[1]))
    a[:, :nin] = X
    a = _r(a, emulate)
    cache = []
    for l, (W, b) in enumerate(layers):
        z = a @ _r(W, emulate).T + b
        cache.append((a, z))
        if l < depth:
            a = _r(np.maximum(z, 0.0), emulate)
    return z[:, :nout], cache


def loss_grad(w, shape, X, T, emulate=False):
    """Mean squared error of the network on (X, T) and its gradient in the flat layout."""
    nin, width, depth, nout = shape
    w = np.asarray(w, dtype=np.float64)
    layers = unpack(w, shape)
    y, cache = forward(w, shape, X, emulate)
    n = X.shape[0]
    e = y - T
    loss = float(np.mean(e * e))
    g = np.zeros_like(w)
    G = unpack(g, shape)
    dz = np.zeros_like(cache[-1][1])
    dz[:, :nout] = 2.0 * e / (n * nout)
    dz = _r(dz, emulate)
    for l in range(depth, -1, -1):
        a, _ = cache[l]
        W, _ = layers[l]
        gW, gb = G[l]
        gW[:] = dz.T @ a
        gb[:] = dz.sum(axis=0)
        if l > 0:
            da = dz @ _r(W, emulate)
            dz = _r(da * (cache[l - 1][1] > 0), emulate)
    return loss, g


def adam_step(w, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam update of (w, m, v) in place; t counts from 1."""
    m[:] = b1 * m + (1 - b1) * g
    v[:] = b2 * v + (1 - b2) * g * g
    w -= lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)


def init_params(shape, seed=0):
    """A random parameter vector with zero padding (for tests; not the CUDA initialiser)."""
    rng = np.random.default_rng(seed)
    lay, n = layout(*shape)
    w = np.zeros(n)
    nin, width, depth, nout = shape
    for l, (W, b) in enumerate(unpack(w, shape)):
        rin = nin if l == 0 else width
        rout = width if l < depth else nout
        s = np.sqrt(6.0 / (rin + rout))
        W[:rout, :rin] = rng.uniform(-s, s, (rout, rin))
        b[:rout] = rng.uniform(-0.1, 0.1, rout)
    return w


# ---------------- features ----------------


def _geometry(verts, tris):
    u, v, w = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    c = (u + v + w) / 3.0
    cr = np.cross(v - u, w - u)
    two_a = np.linalg.norm(cr, axis=1)
    return c, cr / two_a[:, None], 0.5 * two_a


def features(mesh, eps_in, x=None, eps_out=80.0, kappa=0.1257):
    """Per-element features (nt x 18), the 20 normalisers, and the targets (nt x 2) if x given.

    With r the distance from the centroid c_i to charge k, the columns are: c_i minus the
    mean charge position over the radius of gyration sqrt(mean |c - centre|^2) (3); the unit
    normal (3); log(A / mean A); 1 - mean n_i . n_j over the other triangles sharing a vertex
    with i; S1 = sum_k q_k / (4 pi eps_in r) and S2 = sum_k q_k d/dn_x 1 / (4 pi eps_in r)
    (eqbim_3/eqbim_4); U = sum_k |q_k| / (4 pi r); the nearest-charge distance / 3;
    sum_k q_k exp(-kappa r) / (4 pi eps_in r); sum_k q_k / (4 pi eps_in sqrt(r^2 + a^2)) for
    a = 4 and a = 8; sum_k exp(-r^2 / 50) / 10; -sum_k q_k n_i . (c_i - x_k) /
    (4 pi eps_in (r^2 + a^2)^(3/2)) for a = 4 and a = 8. S1, S2, U and the five source
    variants are divided by their root mean square over the molecule. Normalisers: [c]
    divides column c ([0] the radius of gyration for columns 0-2, [6] the mean area inside
    the log, 1 where a column is not scaled); [18] = rms S1 * 2 eps_in / (eps_in + eps_out)
    and [19] = rms S2 * 2 eps_out / (eps_in + eps_out) divide phi and dphi into the targets.
    """
    V, T = mesh.verts, mesh.tris
    nt = T.shape[0]
    c, nrm, A = _geometry(V, T)
    centre = mesh.qpos.mean(axis=0) if mesh.q.size else np.zeros(3)
    d = c - centre
    rg = np.sqrt(np.mean(np.sum(d * d, axis=1)))
    # triangles sharing a vertex (plain sets; small meshes only)
    vt = [[] for _ in range(V.shape[0])]
    for i, t in enumerate(T):
        for a in t:
            vt[a].append(i)
    curv = np.zeros(nt)
    for i, t in enumerate(T):
        nb = set(vt[t[0]]) | set(vt[t[1]]) | set(vt[t[2]])
        nb.discard(i)
        if nb:
            curv[i] = 1.0 - np.mean([nrm[i] @ nrm[j] for j in nb])
    cols = {key: np.zeros(nt) for key in ("s1", "s2", "u", "sk", "a4", "a8", "dens", "e4", "e8")}
    dmin = np.full(nt, np.inf)
    for k in range(mesh.q.size):
        r_vec = c - mesh.qpos[k]
        r = np.linalg.norm(r_vec, axis=1)
        qk = mesh.q[k]
        cols["s1"] += qk / (4 * np.pi * eps_in * r)
        cols["s2"] += qk * (-np.sum(nrm * r_vec, axis=1)) / (4 * np.pi * eps_in * r ** 3)
        cols["u"] += abs(qk) / (4 * np.pi * r)
        cols["sk"] += qk * np.exp(-kappa * r) / (4 * np.pi * eps_in * r)
        cols["a4"] += qk / (4 * np.pi * eps_in * np.sqrt(r * r + 16.0))
        cols["a8"] += qk / (4 * np.pi * eps_in * np.sqrt(r * r + 64.0))
        cols["dens"] += np.exp(-r * r / 50.0)
        nd = np.sum(nrm * r_vec, axis=1)
        cols["e4"] += -qk * nd / (4 * np.pi * eps_in * (r * r + 16.0) ** 1.5)
        cols["e8"] += -qk * nd / (4 * np.pi * eps_in * (r * r + 64.0) ** 1.5)
        dmin = np.minimum(dmin, r)
    rms = lambda a: np.sqrt(np.mean(a * a))  # noqa: E731
    sc = np.ones(NSTAT)
    sc[0], sc[6] = rg, A.mean()
    F = np.zeros((nt, NFEAT))
    F[:, 0:3] = d / rg
    F[:, 3:6] = nrm
    F[:, 6] = np.log(A / sc[6])
    F[:, 7] = curv
    for col, key in ((8, "s1"), (9, "s2"), (10, "u"), (12, "sk"), (13, "a4"), (14, "a8"), (16, "e4"), (17, "e8")):
        sc[col] = rms(cols[key])
        F[:, col] = cols[key] / sc[col]
    F[:, 11] = dmin / 3.0
    F[:, 15] = cols["dens"] / 10.0
    sc[18] = sc[8] * 2 * eps_in / (eps_in + eps_out)
    sc[19] = sc[9] * 2 * eps_out / (eps_in + eps_out)
    Tg = None
    if x is not None:
        Tg = np.stack([x[:nt] / sc[18], x[nt:] / sc[19]], axis=1)
    return F, sc, Tg
