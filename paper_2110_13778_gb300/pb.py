"""Thin ctypes binding of libpb (include/pb.h): argument marshalling only.

Every function keeps the C name. Device arrays are passed as torch CUDA tensors (float64,
contiguous) or raw integer device addresses; host arrays as numpy arrays. Errors raise
``PBError`` with the library's one-line reason. There is no fallback: if libpb.so is not
built, importing this module's functions raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpb.so")

(PB_OK, PB_ERR_ARG, PB_ERR_MESH, PB_ERR_CUDA, PB_ERR_NOT_CONVERGED, PB_ERR_NONFINITE, PB_ERR_STATE, PB_ERR_NOMEM,
 PB_ERR_TIMEOUT) = range(9)
PB_FP64, PB_MIXED = 0, 1
PB_PRECOND_NONE, PB_PRECOND_DIAG, PB_PRECOND_BLOCK = 0, 1, 2
PB_SINGULAR_AUTO, PB_SINGULAR_FP64, PB_SINGULAR_FF = 0, 1, 2
PB_BASIS_CONSTANT, PB_BASIS_LINEAR = 0, 1

EXPORTS = [
    "pb_create", "pb_destroy", "pb_last_error", "pb_mesh_upload", "pb_set_charges", "pb_build_tree",
    "pb_matvec", "pb_rhs", "pb_precond_apply", "pb_gmres_solve", "pb_solvation_energy",
    "pb_get_tree_stats", "pb_get_tree", "pb_matvec_part", "pb_set_timing", "pb_get_timing",
    "pb_get_launch_count", "pb_solvation_energy_noalloc", "pb_solve_states",
    "pb_mlp_create", "pb_mlp_destroy", "pb_mlp_last_error", "pb_mlp_param_count", "pb_mlp_get_params",
    "pb_mlp_set_params", "pb_mlp_forward", "pb_mlp_gradient", "pb_mlp_train_step", "pb_features",
    "pb_learned_guess", "pb_measure_alu_peaks", "pb_autotune", "pb_matvec_multi", "pb_get_graph_launches",
    "pb_solvation_energy_treecode", "pb_batch_solve_states",
]
PB_MAX_RHS = 64
NFEAT = 18
NSTAT = 20


class PBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libpb error {code}: {msg}")
        self.code = code


class pb_params(ctypes.Structure):
    _fields_ = [
        ("eps_in", ctypes.c_double), ("eps_out", ctypes.c_double), ("kappa", ctypes.c_double),
        ("eta0", ctypes.c_double), ("leaf_size", ctypes.c_int), ("levels", ctypes.c_int),
        ("p", ctypes.c_int), ("adaptive", ctypes.c_int), ("qs", ctypes.c_int),
        ("precision", ctypes.c_int), ("precond", ctypes.c_int), ("singular", ctypes.c_int),
        ("pc_block", ctypes.c_int), ("qr", ctypes.c_int), ("basis", ctypes.c_int),
    ]


class pb_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("matvecs", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("status", ctypes.c_int), ("initial_residual", ctypes.c_double)]


class pb_tune_result(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int), ("p", ctypes.c_int), ("matvec_ms", ctypes.c_double),
                ("build_ms", ctypes.c_double), ("rel_err", ctypes.c_double), ("tried", ctypes.c_int),
                ("met_tolerance", ctypes.c_int), ("order", ctypes.c_int * 11)]


class pb_tree_stats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int), ("nclusters", ctypes.c_int * 11), ("nnear", ctypes.c_longlong * 11),
        ("ninter", ctypes.c_longlong * 11), ("order", ctypes.c_int * 11), ("near_pairs", ctypes.c_longlong),
        ("touching", ctypes.c_longlong), ("max_leaf", ctypes.c_int), ("touch_class", ctypes.c_longlong * 4),
        ("pc_blocks", ctypes.c_int), ("pc_max", ctypes.c_int), ("pc_sum_m3", ctypes.c_double),
    ]


_lib = None


def lib():
    """Load libpb.so (built by ``paper_2110_13778_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built: run paper_2110_13778_gb300.build.build() (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        L.pb_create.argtypes = [ctypes.POINTER(pb_params), vp, ctypes.POINTER(vp)]
        L.pb_destroy.argtypes = [vp]
        L.pb_last_error.argtypes = [vp]
        L.pb_last_error.restype = ctypes.c_char_p
        L.pb_mesh_upload.argtypes = [vp, dp, c_int, ip, c_int, dp, dp, c_int]
        L.pb_set_charges.argtypes = [vp, dp, c_int]
        L.pb_build_tree.argtypes = [vp]
        L.pb_matvec.argtypes = [vp, vp, vp]
        L.pb_matvec_part.argtypes = [vp, vp, vp, c_int]
        L.pb_rhs.argtypes = [vp, vp]
        L.pb_precond_apply.argtypes = [vp, vp, vp]
        L.pb_gmres_solve.argtypes = [vp, vp, c_double, c_int, c_int, c_int, ctypes.POINTER(pb_solve_info)]
        L.pb_solvation_energy.argtypes = [vp, vp, dp]
        L.pb_solvation_energy_treecode.argtypes = [vp, vp, c_double, dp]
        L.pb_batch_solve_states.argtypes = [ctypes.POINTER(vp), c_int, ctypes.POINTER(dp), c_int,
                                            ctypes.POINTER(vp), dp, c_double, c_int, c_int,
                                            ctypes.POINTER(pb_solve_info)]
        L.pb_solve_states.argtypes = [vp, dp, c_int, vp, dp, c_double, c_int, c_int, c_int,
                                      ctypes.POINTER(pb_solve_info)]
        L.pb_get_tree_stats.argtypes = [vp, ctypes.POINTER(pb_tree_stats)]
        L.pb_get_tree.argtypes = [vp, ip, ip, ip, ip, ip, ip]
        L.pb_set_timing.argtypes = [vp, c_int]
        L.pb_get_timing.argtypes = [vp, dp]
        L.pb_get_launch_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
        L.pb_solvation_energy_noalloc.argtypes = [vp, vp, c_int, vp, vp, c_int, c_double, c_double, c_double, c_int,
                                                  vp, vp, vp, ctypes.c_char_p, c_int]
        fp = ctypes.POINTER(ctypes.c_float)
        L.pb_mlp_create.argtypes = [c_int, c_int, c_int, c_int, ctypes.c_ulonglong, vp, ctypes.POINTER(vp)]
        L.pb_mlp_destroy.argtypes = [vp]
        L.pb_mlp_last_error.argtypes = [vp]
        L.pb_mlp_last_error.restype = ctypes.c_char_p
        L.pb_mlp_param_count.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
        L.pb_mlp_get_params.argtypes = [vp, fp]
        L.pb_mlp_set_params.argtypes = [vp, fp]
        L.pb_mlp_forward.argtypes = [vp, vp, c_int, vp]
        L.pb_mlp_gradient.argtypes = [vp, vp, vp, c_int, fp, fp]
        L.pb_mlp_train_step.argtypes = [vp, vp, vp, c_int, ctypes.c_float, fp]
        L.pb_features.argtypes = [vp, vp, vp, vp, dp]
        L.pb_learned_guess.argtypes = [vp, vp, vp]
        L.pb_measure_alu_peaks.argtypes = [vp, dp, dp]
        L.pb_matvec_multi.argtypes = [vp, vp, vp, c_int]
        L.pb_get_graph_launches.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
        L.pb_autotune.argtypes = [vp, c_double, c_int, c_int, ctypes.POINTER(pb_tune_result)]
        _lib = L
    return _lib


def _ptr(t):
    """Device address of a contiguous CUDA torch tensor, an int address, or NULL for None."""
    if t is None:
        return ctypes.c_void_p(None)
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check(ctx, rc):
    if rc != PB_OK:
        raise PBError(rc, lib().pb_last_error(ctx).decode())


def params(eps_in=1.0, eps_out=80.0, kappa=0.1257, eta0=0.8, leaf_size=64, levels=0, p=8, adaptive=0, qs=3,
           precision=PB_FP64, precond=PB_PRECOND_BLOCK, singular=0, pc_block=0, qr=0, basis=0):
    return pb_params(eps_in, eps_out, kappa, eta0, leaf_size, levels, p, adaptive, qs, precision, precond, singular,
                     pc_block, qr, basis)


def pb_create(prm: pb_params, stream=0):
    h = ctypes.c_void_p()
    rc = lib().pb_create(ctypes.byref(prm), ctypes.c_void_p(stream), ctypes.byref(h))
    if rc != PB_OK:
        raise PBError(rc, "pb_create rejected the parameters")
    return h


def pb_destroy(ctx):
    lib().pb_destroy(ctx)


def pb_mesh_upload(ctx, verts, tris, qpos, q):
    V = np.ascontiguousarray(verts, dtype=np.float64)
    T = np.ascontiguousarray(tris, dtype=np.int32)
    QP = np.ascontiguousarray(np.reshape(qpos, (-1, 3)), dtype=np.float64)
    Q = np.ascontiguousarray(np.reshape(q, (-1,)), dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(ctx, lib().pb_mesh_upload(ctx, V.ctypes.data_as(dp), V.shape[0], T.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     T.shape[0], QP.ctypes.data_as(dp), Q.ctypes.data_as(dp), Q.shape[0]))


def pb_set_charges(ctx, q):
    Q = np.ascontiguousarray(np.reshape(q, (-1,)), dtype=np.float64)
    _check(ctx, lib().pb_set_charges(ctx, Q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), Q.shape[0]))


def pb_build_tree(ctx):
    _check(ctx, lib().pb_build_tree(ctx))


def pb_matvec(ctx, x, y):
    _check(ctx, lib().pb_matvec(ctx, _ptr(x), _ptr(y)))


def pb_matvec_multi(ctx, X, Y):
    """Y[q] = A X[q] for the rows of X (nr, 2N) float64 CUDA; Y the same shape."""
    _check(ctx, lib().pb_matvec_multi(ctx, _ptr(X), _ptr(Y), int(X.shape[0])))


def pb_matvec_part(ctx, x, y, which):
    _check(ctx, lib().pb_matvec_part(ctx, _ptr(x), _ptr(y), which))


def pb_rhs(ctx, b):
    _check(ctx, lib().pb_rhs(ctx, _ptr(b)))


def pb_precond_apply(ctx, r, z):
    _check(ctx, lib().pb_precond_apply(ctx, _ptr(r), _ptr(z)))


def pb_gmres_solve(ctx, x, tol=1e-6, max_iter=200, restart=50, use_x0=False, raise_on_fail=True):
    info = pb_solve_info()
    rc = lib().pb_gmres_solve(ctx, _ptr(x), tol, max_iter, restart, int(bool(use_x0)), ctypes.byref(info))
    if rc != PB_OK and (raise_on_fail or rc not in (PB_ERR_NOT_CONVERGED, PB_ERR_NONFINITE)):
        _check(ctx, rc)
    return info


def pb_solve_states(ctx, q_states, X, tol=1e-6, max_iter=200, restart=50, warm=True, raise_on_fail=True):
    """Solve nrhs charge states on one built mesh. q_states: (nrhs, nc) host array;
    X: (nrhs, 2N) float64 CUDA tensor (overwritten). warm: False / True (sequential, each from
    the previous solution) or 2 (batched lockstep after state 0). Returns (energies, infos)."""
    Q = np.ascontiguousarray(q_states, dtype=np.float64)
    nrhs = Q.shape[0]
    E = np.zeros(nrhs)
    infos = (pb_solve_info * nrhs)()
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib().pb_solve_states(ctx, Q.ctypes.data_as(dp), nrhs, _ptr(X), E.ctypes.data_as(dp), tol, max_iter,
                               restart, 2 if (warm == 2 and not isinstance(warm, bool)) else int(bool(warm)), infos)
    if rc != PB_OK and (raise_on_fail or rc not in (PB_ERR_NOT_CONVERGED, PB_ERR_NONFINITE)):
        _check(ctx, rc)
    return E, list(infos)


def pb_batch_solve_states(ctxs, q_states, X, tol=1e-6, max_iter=200, restart=50, raise_on_fail=True):
    """Several molecules x several charge states in one graph launch. ctxs: built contexts;
    q_states: per molecule an (nrhs, nc) host array (same nrhs for all); X: per molecule an
    (nrhs, 2N) float64 CUDA tensor (overwritten). Returns (energies (nmol, nrhs), infos as a
    list of per-molecule lists)."""
    nmol = len(ctxs)
    Qs = [np.ascontiguousarray(q, dtype=np.float64) for q in q_states]
    nrhs = Qs[0].shape[0]
    dp = ctypes.POINTER(ctypes.c_double)
    carr = (ctypes.c_void_p * nmol)(*[c.value for c in ctxs])
    qarr = (dp * nmol)(*[q.ctypes.data_as(dp) for q in Qs])
    xarr = (ctypes.c_void_p * nmol)(*[_ptr(x).value for x in X])
    E = np.zeros((nmol, nrhs))
    infos = (pb_solve_info * (nmol * nrhs))()
    rc = lib().pb_batch_solve_states(carr, nmol, qarr, nrhs, xarr, E.ctypes.data_as(dp), tol, max_iter, restart, infos)
    if rc != PB_OK and (raise_on_fail or rc not in (PB_ERR_NOT_CONVERGED, PB_ERR_NONFINITE)):
        _check(ctxs[0], rc)
    inf = list(infos)
    return E, [inf[k * nrhs:(k + 1) * nrhs] for k in range(nmol)]


def pb_solvation_energy(ctx, x):
    E = ctypes.c_double()
    _check(ctx, lib().pb_solvation_energy(ctx, _ptr(x), ctypes.byref(E)))
    return E.value


def pb_solvation_energy_treecode(ctx, x, theta=0.5):
    E = ctypes.c_double()
    _check(ctx, lib().pb_solvation_energy_treecode(ctx, _ptr(x), float(theta), ctypes.byref(E)))
    return E.value


def pb_get_tree_stats(ctx):
    s = pb_tree_stats()
    _check(ctx, lib().pb_get_tree_stats(ctx, ctypes.byref(s)))
    L = s.levels
    return {
        "levels": L,
        "nclusters": list(s.nclusters[: L + 1]),
        "nnear": list(s.nnear[: L + 1]),
        "ninter": list(s.ninter[: L + 1]),
        "order": list(s.order[: L + 1]),
        "near_pairs": s.near_pairs,
        "touching": s.touching,
        "touch_class": list(s.touch_class),
        "max_leaf": s.max_leaf,
        "pc_blocks": s.pc_blocks,
        "pc_max": s.pc_max,
        "pc_sum_m3": s.pc_sum_m3,
    }


def pb_get_tree(ctx, nt):
    st = pb_get_tree_stats(ctx)
    ncl = sum(st["nclusters"])
    order = np.zeros(nt, dtype=np.int32)
    lb = np.zeros(ncl, dtype=np.int32)
    nc = np.zeros(ncl, dtype=np.int32)
    ni = np.zeros(max(1, sum(st["nnear"])), dtype=np.int32)
    ic = np.zeros(ncl, dtype=np.int32)
    ii = np.zeros(max(1, sum(st["ninter"])), dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    _check(ctx, lib().pb_get_tree(ctx, order.ctypes.data_as(ip), lb.ctypes.data_as(ip), nc.ctypes.data_as(ip),
                                  ni.ctypes.data_as(ip), ic.ctypes.data_as(ip), ii.ctypes.data_as(ip)))
    return st, order, lb, nc, ni, ic, ii


def pb_set_timing(ctx, enable):
    _check(ctx, lib().pb_set_timing(ctx, int(enable)))


TIMING_SLOTS = ["near", "corr", "up", "m2l", "down", "precond", "arnoldi", "singular", "tree", "pcbuild",
                "energy", "rhs", "farsetup"]


def pb_get_timing(ctx):
    """{slot: (total_ms, launches)} since the last read."""
    out = (ctypes.c_double * (2 * len(TIMING_SLOTS)))()
    _check(ctx, lib().pb_get_timing(ctx, out))
    return {s: (out[2 * i], int(out[2 * i + 1])) for i, s in enumerate(TIMING_SLOTS)}


def pb_get_graph_launches(ctx):
    n = ctypes.c_longlong()
    _check(ctx, lib().pb_get_graph_launches(ctx, ctypes.byref(n)))
    return n.value


def pb_get_launch_count(ctx):
    n = ctypes.c_longlong()
    _check(ctx, lib().pb_get_launch_count(ctx, ctypes.byref(n)))
    return n.value


def pb_solvation_energy_noalloc(verts, tris, qpos, q, x, E, eps_in=1.0, eps_out=80.0, kappa=0.1257,
                                precision=PB_FP64, stream=0):
    """Energy from caller-owned device tensors into the device scalar E; allocates nothing.
    verts (nv, 3) float64, tris (nt, 3) int32, qpos (nc, 3) float64, q (nc,) float64,
    x (2 nt,) float64, E (1,) float64 -- all contiguous CUDA tensors."""
    err = ctypes.create_string_buffer(256)
    nt = int(tris.shape[0])
    nc = int(q.shape[0])
    rc = lib().pb_solvation_energy_noalloc(_ptr(verts), _ptr(tris), nt, _ptr(qpos), _ptr(q), nc, eps_in, eps_out,
                                           kappa, precision, _ptr(x), _ptr(E), ctypes.c_void_p(stream), err, 256)
    if rc != PB_OK:
        raise PBError(rc, err.value.decode())


# ---------------- learned warm start ----------------


def _mcheck(net, rc):
    if rc != PB_OK:
        raise PBError(rc, lib().pb_mlp_last_error(net).decode())


def pb_mlp_create(nin=NFEAT, width=128, depth=3, nout=2, seed=0, stream=0):
    h = ctypes.c_void_p()
    rc = lib().pb_mlp_create(nin, width, depth, nout, seed, ctypes.c_void_p(stream), ctypes.byref(h))
    if rc != PB_OK:
        raise PBError(rc, "pb_mlp_create rejected the shape or could not allocate")
    return h


def pb_mlp_destroy(net):
    lib().pb_mlp_destroy(net)


def pb_mlp_param_count(net):
    n = ctypes.c_longlong()
    _mcheck(net, lib().pb_mlp_param_count(net, ctypes.byref(n)))
    return n.value


def pb_mlp_get_params(net):
    w = np.zeros(pb_mlp_param_count(net), dtype=np.float32)
    _mcheck(net, lib().pb_mlp_get_params(net, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return w


def pb_mlp_set_params(net, w):
    W = np.ascontiguousarray(w, dtype=np.float32)
    if W.size != pb_mlp_param_count(net):
        raise ValueError("parameter vector has the wrong length")
    _mcheck(net, lib().pb_mlp_set_params(net, W.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))


def pb_mlp_forward(net, X, Y):
    """Y (n, nout) float32 CUDA = network(X (n, nin) float32 CUDA)."""
    _mcheck(net, lib().pb_mlp_forward(net, _ptr(X), int(X.shape[0]), _ptr(Y)))


def pb_mlp_gradient(net, X, T):
    """(loss, gradient as a float32 numpy array) for the batch (X, T)."""
    loss = ctypes.c_float()
    g = np.zeros(pb_mlp_param_count(net), dtype=np.float32)
    _mcheck(net, lib().pb_mlp_gradient(net, _ptr(X), _ptr(T), int(X.shape[0]), ctypes.byref(loss),
                                       g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return loss.value, g


def pb_mlp_train_step(net, X, T, lr=1e-3, want_loss=True):
    loss = ctypes.c_float()
    _mcheck(net, lib().pb_mlp_train_step(net, _ptr(X), _ptr(T), int(X.shape[0]), lr,
                                         ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def pb_features(ctx, F, x=None, T=None):
    """F (nt, 18) float32 CUDA; optional training targets T (nt, 2) float32 CUDA from a
    solution x (2 nt) float64 CUDA. Returns the 20 normalisers."""
    sc = np.zeros(NSTAT)
    _check(ctx, lib().pb_features(ctx, _ptr(F), _ptr(x), _ptr(T), sc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return sc


def pb_learned_guess(ctx, net, x):
    _check(ctx, lib().pb_learned_guess(ctx, net, _ptr(x)))


def pb_measure_alu_peaks(stream=0):
    """(FP32, FP64) FMA throughput of the current device in TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = lib().pb_measure_alu_peaks(ctypes.c_void_p(stream), ctypes.byref(a), ctypes.byref(b))
    if rc != PB_OK:
        raise PBError(rc, "pb_measure_alu_peaks failed")
    return a.value, b.value


def pb_autotune(ctx, tol=1e-4, matvecs_per_solve=10, nrhs=1):
    """Choose leaf size and per-level orders for the uploaded molecule, timing products of
    nrhs vectors; leaves ctx built with them."""
    r = pb_tune_result()
    _check(ctx, lib().pb_autotune(ctx, tol, matvecs_per_solve, nrhs, ctypes.byref(r)))
    out = {f: getattr(r, f) for f, _ in pb_tune_result._fields_}
    out["order"] = list(r.order)
    return out
