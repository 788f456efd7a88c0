"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only builds inputs (meshes, charges, vectors). It holds none of the method's
arithmetic, so the CUDA path and the CPU oracle can both draw from it without sharing code.

* ``icosphere(level, radius)`` -- the geodesic sphere the Kirkwood tests use (Section 3.1):
  an icosahedron whose faces are split into four by edge midpoints ``level`` times, every
  new vertex pushed out to the sphere. It has ``20 * 4**level`` flat triangles with welded
  vertices, listed counter-clockwise seen from outside (so ``(v-u) x (w-u)`` points out).
* ``ball_charges(n, r, seed)`` -- ``n`` point charges uniform in a ball of radius ``r``
  (radius ``r u**(1/3)``, isotropic direction), values uniform in [-1, 1].
* ``random_density(n, seed)`` -- a seeded vector ``[phi; dphi/dn]`` for matvec tests.
"""
from __future__ import annotations

import numpy as np

__all__ = ["Mesh", "icosphere", "ball_charges", "random_density", "perturbed_sphere"]


class Mesh:
    """Triangulated surface with point charges.

    verts: float64 (nv, 3); tris: int32 (nt, 3), counter-clockwise seen from outside;
    qpos: float64 (nc, 3); q: float64 (nc,) charges in units of e.
    """

    def __init__(self, verts, tris, qpos, q):
        self.verts = np.ascontiguousarray(verts, dtype=np.float64)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.qpos = np.ascontiguousarray(np.reshape(qpos, (-1, 3)), dtype=np.float64)
        self.q = np.ascontiguousarray(np.reshape(q, (-1,)), dtype=np.float64)

    @property
    def nt(self) -> int:
        return int(self.tris.shape[0])

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nc(self) -> int:
        return int(self.q.shape[0])


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
         [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]],
        dtype=np.float64,
    )
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]],
        dtype=np.int64,
    )
    return v / np.linalg.norm(v, axis=1, keepdims=True), f


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Return (verts, tris) of the level-``level`` geodesic sphere."""
    v, f = _icosahedron()
    verts = [row for row in v]
    for _ in range(level):
        cache = {}
        new_f = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                m = verts[a] + verts[b]
                m = m / np.linalg.norm(m)
                verts.append(m)
                idx = len(verts) - 1
                cache[key] = idx
            return idx

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_f += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = np.array(new_f, dtype=np.int64)
    V = np.array(verts, dtype=np.float64) * radius + np.asarray(center, dtype=np.float64)
    # orient counter-clockwise seen from outside
    P = V[f]
    nrm = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    outward = np.einsum("ij,ij->i", nrm, P.mean(axis=1) - np.asarray(center)) > 0
    f = np.where(outward[:, None], f, f[:, [0, 2, 1]])
    return V, f.astype(np.int32)


def perturbed_sphere(level: int, radius: float, amp: float, seed: int):
    """Icosphere with vertices moved radially by a smooth seeded bump field (irregular
    element sizes and shapes, still closed and outward oriented for amp < 0.3 radius)."""
    V, T = icosphere(level, 1.0)
    rng = np.random.Generator(np.random.PCG64(seed))
    dirs = rng.normal(size=(6, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    w = rng.uniform(0.5, 1.0, size=6)
    bump = np.zeros(V.shape[0])
    for k in range(6):
        bump += w[k] * np.exp(-4.0 * (1.0 - V @ dirs[k]))
    V = V * (radius * (1.0 + amp * (bump - bump.mean())))[:, None]
    return V, T


def ball_charges(n: int, r: float, seed: int):
    """n charges uniform in the ball of radius r with values uniform in [-1, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = r * rng.uniform(0.0, 1.0, size=n) ** (1.0 / 3.0)
    q = rng.uniform(-1.0, 1.0, size=n)
    return d * rad[:, None], q


def random_density(nt: int, seed: int):
    """Seeded [phi; dphi/dn] test vector of length 2*nt with values in [-1, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=2 * nt)


def kirkwood_centered(level: int, radius: float, q: float = 1.0):
    V, T = icosphere(level, radius)
    return Mesh(V, T, np.zeros((1, 3)), np.array([q]))


def kirkwood_ball(level: int, radius: float, nq: int, rq: float, seed: int):
    V, T = icosphere(level, radius)
    qp, q = ball_charges(nq, rq, seed)
    return Mesh(V, T, qp, q)
