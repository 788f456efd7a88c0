"""Synthetic protein-like molecules: the walk's constraints and the surface's topology. CPU."""
from collections import Counter

import numpy as np
import pytest

from paper_2110_13778_gb300 import molecules


def test_saw_constraints():
    pos, rad, q = molecules.saw_atoms(300, seed=11)
    steps = np.linalg.norm(np.diff(pos, axis=0), axis=1)
    assert np.allclose(steps, 1.5)
    d = np.linalg.norm(pos[:, None] - pos[None], axis=2)
    i, j = np.triu_indices(len(pos), 2)
    assert d[i, j].min() >= 2.8 - 1e-12
    assert set(np.unique(rad)) <= set(molecules.RADII)
    assert abs(q.sum() - round(q.sum())) < 1e-9
    assert np.all(np.abs(q - (q.sum() - round(q.sum())) / len(q)) <= 0.8 + 1.0 / len(q))


@pytest.mark.parametrize("n,seed,h", [(30, 5, 1.0), (60, 6, 0.8)])
def test_surface_closed_manifold_outward(n, seed, h):
    m, rad = molecules.molecule(n, seed, h)
    V, T = m.verts, m.tris
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    directed = set(map(tuple, e))
    # every directed edge has its reverse: closed and consistently oriented
    assert all((b, a) in directed for a, b in e)
    cnt = Counter(tuple(sorted(x)) for x in e)
    assert all(v == 2 for v in cnt.values())
    # outward: positive enclosed volume; all charges inside (winding number 1)
    vol = np.einsum("ij,ij->i", V[T[:, 0]], np.cross(V[T[:, 1]], V[T[:, 2]])).sum() / 6
    assert vol > 0
    P = V[T]
    for x in m.qpos[:: max(1, len(m.qpos) // 7)]:
        R = P - x
        r = np.linalg.norm(R, axis=2)
        num = np.einsum("ij,ij->i", R[:, 0], np.cross(R[:, 1], R[:, 2]))
        den = (r[:, 0] * r[:, 1] * r[:, 2] + np.einsum("ij,ij->i", R[:, 0], R[:, 1]) * r[:, 2]
               + np.einsum("ij,ij->i", R[:, 0], R[:, 2]) * r[:, 1] + np.einsum("ij,ij->i", R[:, 1], R[:, 2]) * r[:, 0])
        wind = (2 * np.arctan2(num, den)).sum() / (4 * np.pi)
        assert abs(wind - 1.0) < 1e-6


def test_clean_mesh_keeps_a_closed_oriented_surface():
    from oracle import dense

    raw = molecules.molecule(60, 3060, 0.9)[0]
    m = molecules.molecule(60, 3060, 0.9, clean=True)[0]
    assert m.nt < raw.nt
    T = m.tris.astype(np.int64)
    nv = len(m.verts)
    E = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    d = E[:, 0] * nv + E[:, 1]
    r = E[:, 1] * nv + E[:, 0]
    # closed and consistently oriented: every directed edge once, its reverse once
    assert len(np.unique(d)) == len(d) and np.array_equal(np.sort(d), np.sort(r))
    # Euler characteristic unchanged (edge collapses keep the topology)
    def chi(mm):
        TT = mm.tris.astype(np.int64)
        EE = np.unique(np.sort(np.concatenate([TT[:, [0, 1]], TT[:, [1, 2]], TT[:, [2, 0]]]), axis=1), axis=0)
        return len(np.unique(TT)) - len(EE) + len(TT)
    assert chi(m) == chi(raw)
    # the tiny triangles are gone; the enclosed volume barely moves
    _, a_raw, _ = dense.geometry(raw.verts, raw.tris)
    c, a, n = dense.geometry(m.verts, m.tris)
    assert (a / a.mean() < 1e-4).sum() < 0.1 * (a_raw / a_raw.mean() < 1e-4).sum()
    vol = lambda mm: np.sum(np.einsum("ij,ij->i", dense.geometry(mm.verts, mm.tris)[0], dense.geometry(mm.verts, mm.tris)[2]) * dense.geometry(mm.verts, mm.tris)[1]) / 3
    assert abs(vol(m) - vol(raw)) < 2e-3 * vol(raw)
