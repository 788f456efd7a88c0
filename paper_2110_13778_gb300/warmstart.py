"""Learned warm start for GMRES: dataset generation, training and use.

The network (18 features -> 128 -> 128 -> 128 -> 2, ReLU, BF16 tensor-core kernels with
FP32 accumulation) is trained on solutions the solver itself produces: every training
molecule is solved by GMRES from a zero start, and its per-element features and scaled
solution become rows of the training set. At use, ``pb_learned_guess`` evaluates the
network on a new molecule and GMRES starts from the prediction; GMRES to the requested
residual remains the judge, so a poor prediction costs iterations, never accuracy.

Everything here is marshalling around the C ABI: the solves, the features, the forward and
backward passes and the Adam steps all run in libpb's kernels; torch only holds the device
buffers.
"""
from __future__ import annotations

import time

import numpy as np

from . import molecules, pb

WIDTH, DEPTH = 128, 3


def solve_params(**kw):
    base = dict(leaf_size=32, eta0=0.7, p=6, precision=pb.PB_MIXED, precond=pb.PB_PRECOND_BLOCK)
    base.update(kw)
    return pb.params(**base)


def training_rows(mesh, prm, tol=1e-6, max_iter=1000, restart=200):
    """(F, T, info) for one molecule: features (nt, 18) and targets (nt, 2) as float32 CUDA
    tensors from its GMRES solution."""
    import torch

    ctx = pb.pb_create(prm)
    try:
        pb.pb_mesh_upload(ctx, mesh.verts, mesh.tris, mesh.qpos, mesh.q)
        pb.pb_build_tree(ctx)
        x = torch.zeros(2 * mesh.nt, device="cuda", dtype=torch.float64)
        info = pb.pb_gmres_solve(ctx, x, tol=tol, max_iter=max_iter, restart=restart)
        F = torch.empty((mesh.nt, pb.NFEAT), device="cuda", dtype=torch.float32)
        T = torch.empty((mesh.nt, 2), device="cuda", dtype=torch.float32)
        pb.pb_features(ctx, F, x, T)
        torch.cuda.synchronize()
        return F, T, info
    finally:
        pb.pb_destroy(ctx)


def make_dataset(atom_counts, seed=0, grid=1.0, prm=None, clean=False):
    """Features and targets of freshly generated molecules (atom counts as given, seeded;
    clean: collapse the short edges of their surfaces), concatenated and shuffled once by a
    seeded row permutation."""
    import torch

    prm = prm or solve_params()
    Fs, Ts = [], []
    for i, n in enumerate(atom_counts):
        mesh, _ = molecules.molecule(int(n), seed + 1009 * i, grid, clean=clean)
        F, T, _ = training_rows(mesh, prm)
        Fs.append(F)
        Ts.append(T)
    F = torch.cat(Fs)
    T = torch.cat(Ts)
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(F.shape[0])).to(F.device)
    return F.index_select(0, perm).contiguous(), T.index_select(0, perm).contiguous()


def train(net, F, T, steps=2000, batch=4096, lr=2e-3, lr_final=2e-4, log_every=0):
    """Adam on contiguous mini-batches cycled through the (pre-shuffled) rows, learning rate
    decaying geometrically from lr to lr_final. Returns (first loss, last loss, seconds)."""
    import torch

    n = F.shape[0]
    batch = min(batch, n)
    nb = max(1, n // batch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    first = last = None
    for s in range(steps):
        b = s % nb
        Xb = F[b * batch:(b + 1) * batch]
        Tb = T[b * batch:(b + 1) * batch]
        a = lr * (lr_final / lr) ** (s / max(1, steps - 1))
        want = s == 0 or s == steps - 1 or (log_every and s % log_every == 0)
        loss = pb.pb_mlp_train_step(net, Xb, Tb, a, want_loss=bool(want))
        if s == 0:
            first = loss
        if want:
            last = loss
            if log_every:
                print(f"step {s} loss {loss:.4e}")
    torch.cuda.synchronize()
    return first, last, time.perf_counter() - t0


def evaluate(net, mesh, prm, tol=1e-6, max_iter=300, restart=50):
    """Solve one molecule from zero and from the learned guess.

    Returns dict with both infos, both energies and the device times of the two solves
    (the learned one includes the network's inference)."""
    import torch

    out = {}
    ctx = pb.pb_create(prm)
    try:
        pb.pb_mesh_upload(ctx, mesh.verts, mesh.tris, mesh.qpos, mesh.q)
        pb.pb_build_tree(ctx)
        for mode in ("zero", "learned"):
            x = torch.zeros(2 * mesh.nt, device="cuda", dtype=torch.float64)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if mode == "learned":
                pb.pb_learned_guess(ctx, net, x)
            info = pb.pb_gmres_solve(ctx, x, tol=tol, max_iter=max_iter, restart=restart,
                                     use_x0=(mode == "learned"))
            torch.cuda.synchronize()
            out[mode] = dict(info=info, seconds=time.perf_counter() - t0, energy=pb.pb_solvation_energy(ctx, x))
    finally:
        pb.pb_destroy(ctx)
    return out
