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
* ``clean_mesh(V, T, lmin)`` -- collapses edges shorter than lmin where the surface stays a
  closed manifold (the slivers that linear cuts next to grid points leave).
* ``molecule(n, seed, h, clean)`` -- both together as an ``inputs.Mesh``.
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


def clean_mesh(V, T, lmin):
    """Collapse every edge shorter than lmin, shortest first, into its midpoint, where the
    collapse keeps the surface a closed 2-manifold (link condition: the two end vertices share
    exactly the two opposite vertices of the edge's triangles) and turns no neighbouring
    triangle over or to zero area; the edge's two triangles disappear. Linear cuts next to grid
    points leave triangles with areas down to 1e-11 of the mean; these are removed (the
    standard mesh-quality step of isosurface extraction). Returns (V, T, collapses)."""
    nv = len(V)
    E = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]]).astype(np.int64)
    E.sort(axis=1)
    L = np.linalg.norm(V[E[:, 0]] - V[E[:, 1]], axis=1)
    sel = np.flatnonzero(L < lmin)
    if sel.size == 0:
        return V, T, 0
    key, first = np.unique(E[sel, 0] * nv + E[sel, 1], return_index=True)
    sel = sel[first]
    sel = sel[np.argsort(L[sel], kind="stable")]
    cand = E[sel].tolist()
    order = np.argsort(T.reshape(-1), kind="stable")
    tri_of = (order // 3).tolist()
    ptr = np.searchsorted(T.reshape(-1)[order], np.arange(nv + 1)).tolist()
    Vl = V.tolist()
    Tl = T.tolist()
    alive = [True] * len(Tl)
    inc = {}
    dead = set()
    lmin2 = lmin * lmin

    def tris_of(v):
        s_ = inc.get(v)
        if s_ is None:
            s_ = set(tri_of[ptr[v]:ptr[v + 1]])
            inc[v] = s_
        return s_

    def normal(a, b, c):
        ux, uy, uz = b[0] - a[0], b[1] - a[1], b[2] - a[2]
        vx, vy, vz = c[0] - a[0], c[1] - a[1], c[2] - a[2]
        return (uy * vz - uz * vy, uz * vx - ux * vz, ux * vy - uy * vx)

    ncol = 0
    for u, v in cand:
        if u in dead or v in dead:
            continue
        pu, pv = Vl[u], Vl[v]
        if (pu[0] - pv[0]) ** 2 + (pu[1] - pv[1]) ** 2 + (pu[2] - pv[2]) ** 2 >= lmin2:
            continue  # an end moved in an earlier collapse
        tu, tv = tris_of(u), tris_of(v)
        shared = tu & tv
        if len(shared) != 2:
            continue
        opp = set()
        for t in shared:
            opp.update(Tl[t])
        opp.discard(u)
        opp.discard(v)
        nu, nvv = set(), set()
        for t in tu:
            nu.update(Tl[t])
        for t in tv:
            nvv.update(Tl[t])
        nu.discard(u)
        nvv.discard(v)
        if len(opp) != 2 or (nu & nvv) != opp:
            continue
        m = [0.5 * (pu[0] + pv[0]), 0.5 * (pu[1] + pv[1]), 0.5 * (pu[2] + pv[2])]
        ok = True
        for t in (tu | tv) - shared:
            n0 = normal(*[Vl[w] for w in Tl[t]])
            n1 = normal(*[m if w == u or w == v else Vl[w] for w in Tl[t]])
            if n0[0] * n1[0] + n0[1] * n1[1] + n0[2] * n1[2] <= 0.0 or n1[0] ** 2 + n1[1] ** 2 + n1[2] ** 2 <= 1e-24:
                ok = False
                break
        if not ok:
            continue
        Vl[u] = m
        for t in tv - shared:
            Tl[t] = [u if w == v else w for w in Tl[t]]
        for t in shared:
            alive[t] = False
            for w in Tl[t]:
                if w != u and w != v:
                    tris_of(w).discard(t)
        inc[u] = (tu | tv) - shared
        dead.add(v)
        inc.pop(v, None)
        ncol += 1
    Tn = np.array([t for t, a in zip(Tl, alive) if a], dtype=np.int64)
    used, remap = np.unique(Tn.reshape(-1), return_inverse=True)
    return np.array(Vl)[used], remap.reshape(-1, 3).astype(np.int32), ncol


def molecule(n_atoms: int, seed: int, h: float = 0.5, clean: bool = False):
    """The molecule and its surface; clean=True collapses the edges shorter than h / 10
    (clean_mesh)."""
    pos, rad, q = saw_atoms(n_atoms, seed)
    V, T = gaussian_surface(pos, rad, h)
    if clean:
        V, T, _ = clean_mesh(V, T, 0.1 * h)
    return Mesh(V, T, pos, q), rad
