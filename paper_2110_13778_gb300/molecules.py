"""Seeded synthetic protein-like molecules and their triangulated surfaces.

Inputs only (no method arithmetic): used by the tests and the benchmark, and by the oracle
side through the same arrays.

* ``saw_atoms(n, seed)`` -- a self-avoiding random walk of n atoms with step 1.5 A and a
  minimum separation of 2.8 A between atoms at least two apart in the chain; radii drawn from
  {1.2, 1.55, 1.7, 1.8} A with probabilities {0.5, 0.15, 0.3, 0.05}; partial charges uniform in
  [-0.8, 0.8] e, shifted by a common amount so that they sum to the nearest integer.
* ``gaussian_surface(pos, rad, h, iso)`` -- the level set sum_i exp(-(|x - x_i| / r_i)^2) = iso
  on a grid of spacing h, triangulated by marching tetrahedra (six tetrahedra per grid cube
  along the main diagonal, so neighbouring cubes agree on shared faces): a closed, conforming
  (welded), outward-oriented surface.
* ``molecule(n, seed, h)`` -- both together as an ``inputs.Mesh``.
"""
from __future__ import annotations

import numpy as np

from .inputs import Mesh

RADII = np.array([1.2, 1.55, 1.7, 1.8])
RADII_P = np.array([0.5, 0.15, 0.3, 0.05])


def saw_atoms(n: int, seed: int, step: float = 1.5, dmin: float = 2.8, max_tries: int = 200):
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = np.zeros((n, 3))
    cell = dmin
    grid: dict = {}

    def key(p):
        return tuple(np.floor(p / cell).astype(np.int64))

    def ok(p, i):
        k = key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in grid.get((k[0] + dx, k[1] + dy, k[2] + dz), ()):
                        if j < i - 1 and np.sum((pos[j] - p) ** 2) < dmin * dmin:
                            return False
        return True

    grid.setdefault(key(pos[0]), []).append(0)
    i = 1
    backtracks = 0
    while i < n:
        placed = False
        for _ in range(max_tries):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            p = pos[i - 1] + step * d
            if ok(p, i):
                pos[i] = p
                grid.setdefault(key(p), []).append(i)
                placed = True
                break
        if placed:
            i += 1
            continue
        # dead end: take the last few atoms back and regrow them
        backtracks += 1
        if backtracks > 100 * n:
            raise RuntimeError("self-avoiding walk got stuck; try another seed")
        k = min(i - 1, 8)
        for j in range(i - k, i):
            grid[key(pos[j])].remove(j)
        i -= k
    rad = rng.choice(RADII, size=n, p=RADII_P)
    q = rng.uniform(-0.8, 0.8, size=n)
    q += (np.round(q.sum()) - q.sum()) / n
    return pos, rad, q


# the six tetrahedra of the unit cube along the main diagonal (corner index = x + 2y + 4z)
_TETS = np.array([[0, 1, 3, 7], [0, 1, 5, 7], [0, 2, 3, 7], [0, 2, 6, 7], [0, 4, 5, 7], [0, 4, 6, 7]])
_CORNER = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)])  # index = x + 2y + 4z


def _field(pos, rad, h, pad):
    lo = pos.min(0) - pad
    hi = pos.max(0) + pad
    shape = np.ceil((hi - lo) / h).astype(int) + 1
    F = np.zeros(shape, dtype=np.float64)
    cut = 3.0
    for p, r in zip(pos, rad):
        a = np.maximum(np.floor((p - cut * r - lo) / h).astype(int), 0)
        b = np.minimum(np.ceil((p + cut * r - lo) / h).astype(int) + 1, shape)
        xs = lo[0] + h * np.arange(a[0], b[0])
        ys = lo[1] + h * np.arange(a[1], b[1])
        zs = lo[2] + h * np.arange(a[2], b[2])
        d2 = ((xs - p[0]) ** 2)[:, None, None] + ((ys - p[1]) ** 2)[None, :, None] + ((zs - p[2]) ** 2)[None, None, :]
        F[a[0]:b[0], a[1]:b[1], a[2]:b[2]] += np.exp(-d2 / (r * r))
    return F, lo


def gaussian_surface(pos, rad, h=0.5, iso=1.0):
    F, lo = _field(pos, rad, h, pad=3.0 * rad.max())
    iso = iso + 1e-9  # keep grid values off the level set (no zero-length edge cuts)
    inside = F > iso
    nx, ny, nz = F.shape
    # cubes whose corners are not all on one side
    c = np.zeros((nx - 1, ny - 1, nz - 1, 8), dtype=bool)
    for k, (x, y, z) in enumerate(_CORNER):
        c[..., k] = inside[x:nx - 1 + x, y:ny - 1 + y, z:nz - 1 + z]
    mixed = c.any(-1) & ~c.all(-1)
    cubes = np.argwhere(mixed)  # (m, 3) lower corner indices
    tris = []
    for tet in _TETS:
        corners = cubes[:, None, :] + _CORNER[tet][None, :, :]  # (m, 4, 3)
        val = F[corners[..., 0], corners[..., 1], corners[..., 2]]  # (m, 4)
        ins = val > iso
        cnt = ins.sum(1)
        for case_n in (1, 2, 3):
            sel = np.flatnonzero(cnt == case_n)
            if sel.size == 0:
                continue
            cv, cc, ci = val[sel], corners[sel], ins[sel]
            # order the 4 corners so that the inside ones come first (stable)
            order = np.argsort(~ci, axis=1, kind="stable")
            cv = np.take_along_axis(cv, order, 1)
            cc = np.take_along_axis(cc, order[..., None], 1)
            if case_n == 1:
                tris.append(_emit(cv, cc, [(0, 1), (0, 2), (0, 3)], lo, h, iso))
            elif case_n == 3:
                tris.append(_emit(cv, cc, [(0, 3), (1, 3), (2, 3)], lo, h, iso))
            else:
                # inside {0, 1}, outside {2, 3}: the cut is the quad 0-2, 0-3, 1-3, 1-2
                q = [(0, 2), (0, 3), (1, 3), (1, 2)]
                tris.append(_emit(cv, cc, [q[0], q[1], q[2]], lo, h, iso))
                tris.append(_emit(cv, cc, [q[0], q[2], q[3]], lo, h, iso))
    P = np.concatenate([t[0] for t in tris])  # (ntri, 3, 3) vertex positions
    K = np.concatenate([t[1] for t in tris])  # (ntri, 3) edge keys
    G = np.concatenate([t[2] for t in tris])  # (ntri, 3) outward direction (inside -> outside)
    # weld vertices by their grid-edge key
    keys, inv = np.unique(K.reshape(-1), return_inverse=True)
    V = np.zeros((keys.size, 3))
    V[inv] = P.reshape(-1, 3)
    T = inv.reshape(-1, 3).astype(np.int64)
    # orient counter-clockwise seen from outside
    nrm = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, G) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    # drop degenerate triangles (two welded corners)
    good = (T[:, 0] != T[:, 1]) & (T[:, 1] != T[:, 2]) & (T[:, 0] != T[:, 2])
    area2 = np.linalg.norm(np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]), axis=1)
    good &= area2 > 1e-12
    T = T[good]
    used, remap = np.unique(T.reshape(-1), return_inverse=True)
    return V[used], remap.reshape(-1, 3).astype(np.int32)


SNAP = 0.0  # cut points this close to a grid point (in edge fractions) would move onto it (off)


def _emit(cv, cc, edges, lo, h, iso):
    """Triangle vertices on the given tetrahedron edges (corner pairs inside -> outside).
    A cut within SNAP of an end of its edge is moved onto that grid point and keyed by it, so
    every edge meeting at the point shares the vertex; triangles that collapse are dropped
    later. This removes the slivers that linear cuts next to grid points would create."""
    n = cv.shape[0]
    P = np.zeros((n, 3, 3))
    K = np.zeros((n, 3), dtype=np.int64)
    gdir = np.zeros((n, 3))
    for s, (a, b) in enumerate(edges):
        fa, fb = cv[:, a], cv[:, b]
        t = (fa - iso) / (fa - fb)
        pa = lo + h * cc[:, a, :]
        pb = lo + h * cc[:, b, :]
        ka = _gkey(cc[:, a, :])
        kb = _gkey(cc[:, b, :])
        # edge keys live above the grid-point keys, which are < 2^30
        key = (np.minimum(ka, kb) + 1) * (1 << 31) + np.maximum(ka, kb)
        P[:, s, :] = pa + t[:, None] * (pb - pa)
        lo_snap = t < SNAP
        hi_snap = t > 1.0 - SNAP
        P[lo_snap, s, :] = pa[lo_snap]
        P[hi_snap, s, :] = pb[hi_snap]
        key = np.where(lo_snap, ka, np.where(hi_snap, kb, key))
        K[:, s] = key
        gdir += pb - pa  # inside corner -> outside corner
    return P, K, gdir


def _gkey(ijk):
    return (ijk[:, 0].astype(np.int64) * 1024 + ijk[:, 1]) * 1024 + ijk[:, 2]


def molecule(n_atoms: int, seed: int, h: float = 0.5):
    pos, rad, q = saw_atoms(n_atoms, seed)
    V, T = gaussian_surface(pos, rad, h)
    return Mesh(V, T, pos, q), rad
