#!/usr/bin/env python
"""Benchmark of the FMM-accelerated Galerkin PB solve on GB300.

Workload (default): the largest single-GPU configuration -- a 20000-atom synthetic
protein-like molecule (self-avoiding walk, step 1.5 A, minimum separation 2.8 A; radii
{1.2, 1.55, 1.7, 1.8} A; charges U[-0.8, 0.8] e shifted to an integer total; seed 23000)
under the level-1.0 surface of sum_i exp(-(d/r_i)^2) on a 0.9 A grid, edges shorter than
0.09 A collapsed: 1,836,805 flat triangles, 3.67M unknowns, 20000 charges. eps_in = 1,
eps_out = 80, kappa = 0.1257 / A; FMM order p = 8, eta0 = 0.8, leaf size 64, FP32 bulk
arithmetic with float-float singular integrals and FP64 Arnoldi, preconditioner and energy
(mixed precision), block-diagonal preconditioner, GMRES(200) to 1e-6 relative residual,
solvation energy by the Cartesian treecode (theta 0.5). --workload sphere runs the Kirkwood
sphere with off-centre charges (radius 20 A, icosphere level 6, 81920 triangles, 50 charges).

One step = the whole hot path on the resident mesh: pb_build_tree (geometry, octree,
lists, singular integrals, preconditioner), pb_gmres_solve (right-hand side + GMRES with
FMM products) and the solvation energy. value = element-matvecs per second of the step:
N x (matrix-vector products the solver performed) / step time, in Melem/s -- setup
included. Inputs are far larger than the 129 MB L2 (and the L2 is flushed between steps,
outside the timed events). The plain FP64 method is timed on the same molecule in the same
run (fp64_method), and the ratio of the two solve times is reported beside the value.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload sphere]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM matvec Melem/s (whole solve: setup + GMRES to 1e-6 + energy)"
UNIT = "Melem/s"
FLOPS_PER_NEAR_PAIR = 75  # formula count of the near-field pair evaluation (exp, rsqrt as 1 each)


def workload(level=6, seed=2000, kind="molecule", atoms=20000, h=0.9, clean=True):
    """A protein-like molecule (default): a self-avoiding walk of `atoms` atoms under its
    Gaussian isosurface (grid spacing h), edges shorter than h / 10 collapsed unless clean is
    False; or the Kirkwood sphere with off-centre charges."""
    if kind == "molecule":
        from paper_2110_13778_gb300 import molecules

        return molecules.molecule(atoms, 3000 + atoms, h, clean=clean)[0]
    from paper_2110_13778_gb300 import inputs

    return inputs.kirkwood_ball(level, 20.0, 50, 16.0, seed)


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--level", type=int, default=6)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--leaf", type=int, default=64)
    ap.add_argument("--eta0", type=float, default=0.8)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--restart", type=int, default=200, help="GMRES restart length m (Krylov basis vectors)")
    ap.add_argument("--energy", default="treecode", choices=["treecode", "direct"],
                    help="solvation energy of the step: the Cartesian treecode of Section 2.5 or the direct sum")
    ap.add_argument("--theta", type=float, default=0.5, help="treecode MAC parameter")
    ap.add_argument("--workload", default="molecule",
                    choices=["sphere", "molecule", "batch", "learned", "precond", "linear"])
    ap.add_argument("--train-molecules", type=int, default=48)
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--train-atoms", type=int, nargs=2, default=[50, 500], metavar=("MIN", "MAX"),
                    help="training molecules: atom counts log-uniform in [MIN, MAX]")
    ap.add_argument("--atoms", type=int, default=None,
                    help="molecule size (default 20000 for --workload molecule, 2000 for learned and linear)")
    ap.add_argument("--fp64-budget", type=float, default=60.0,
                    help="seconds of timed FP64-method steps (at most --steps of them, at least one)")
    ap.add_argument("--grid", type=float, default=0.9)
    ap.add_argument("--raw-mesh", action="store_true",
                    help="molecules: keep the marching-tetrahedra slivers (no short-edge collapse)")
    ap.add_argument("--molecules", type=int, default=64)
    ap.add_argument("--max-atoms", type=int, default=8000)
    ap.add_argument("--batch-restart", type=int, default=30)
    ap.add_argument("--states", type=int, default=16)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="sphere / molecule: choose leaf size and per-level orders with pb_autotune first (untimed)")
    a = ap.parse_args()
    if a.atoms is None:
        a.atoms = 2000 if a.workload in ("learned", "linear") else 20000
    return a


# ---------------------------------------------------------------- clocks during the timed region
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # nvidia-smi takes a moment to start: the timed region begins after its first sample
            t0 = time.perf_counter()
            while not self.samples and self.proc.poll() is None and time.perf_counter() - t0 < 3.0:
                time.sleep(0.01)
            self.first = len(self.samples)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        # samples taken inside the timed region; the one just before it if the region was shorter
        # than the sampling interval
        inside = self.samples[getattr(self, "first", 0):]
        self.samples = inside if inside else self.samples[-1:]
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        reasons = set()
        for s in self.samples:
            for k, name in enumerate(self.NAMES):
                if s[3 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------- distributed plumbing (replicas)
def dist_setup(ngpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if os.environ.get("PB_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return rank, world, local


def dist_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ---------------------------------------------------------------- CPU oracle baseline
def cpu_oracle_rate(mesh, budget_s=12.0, max_rows=None):
    """Dense-Galerkin rows of A x per second on the host cores (oracle, as it stands).
    A full product is N rows, so rows/s / 1e6 is the oracle's element-matvec rate."""
    from oracle import dense

    ph = dense.Phys(1.0, 80.0, 0.1257, qs=3)
    x = np.random.default_rng(0).uniform(-1, 1, 2 * mesh.nt)
    rows = 8
    t0 = time.perf_counter()
    dense.rows_matvec(mesh.verts, mesh.tris, ph, np.arange(rows), x)
    t1 = time.perf_counter() - t0
    nrows = int(min(mesh.nt if max_rows is None else max_rows, max(rows, budget_s / max(t1, 1e-9) * rows)))
    sel = np.linspace(0, mesh.nt - 1, nrows).astype(np.int32)
    t0 = time.perf_counter()
    dense.rows_matvec(mesh.verts, mesh.tris, ph, sel, x)
    dt = time.perf_counter() - t0
    return nrows / dt / 1e6, nrows, dt


def run_reference(a):
    rank, world, local = dist_setup(a.gpus)
    if rank != 0:
        return 0
    mesh = workload(a.level, kind=a.workload if a.workload in ("sphere", "molecule") else "molecule", atoms=a.atoms,
                    h=a.grid, clean=not a.raw_mesh)
    cores = os.cpu_count()
    for _ in range(a.warmup):
        cpu_oracle_rate(mesh, budget_s=1.0, max_rows=64)
    vals, times = [], []
    for _ in range(a.steps):
        v, nrows, dt = cpu_oracle_rate(mesh, budget_s=8.0)
        vals.append(v)
        times.append(dt)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(a, mesh),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"dense Galerkin rows of A x (one-point + Sauter-Schwab qs=3), {nrows} sampled rows "
                                   f"of the {mesh.nt}-triangle workload per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def config_dict(a, mesh):
    if a.workload == "molecule":
        wl = (f"protein-like molecule: {a.atoms}-atom self-avoiding walk, Gaussian isosurface at 1.0 on a "
              f"{a.grid} A grid, " + ("" if a.raw_mesh else f"edges < {a.grid / 10:.2f} A collapsed, ") +
              f"{mesh.nt} triangles, {mesh.nc} charges, eps 1/80, kappa 0.1257")
    else:
        wl = (f"Kirkwood sphere r=20 A, icosphere level {a.level} ({mesh.nt} triangles), 50 charges in r<=16 A, "
              f"eps 1/80, kappa 0.1257")
    return {
        "workload": wl,
        "N": mesh.nt, "p": a.p, "eta0": a.eta0, "leaf_size": a.leaf, "precision": a.precision,
        "precond": "block-diagonal (leaf level)", "gmres": f"GMRES({a.restart}) tol {a.tol}",
        "step": "build_tree + gmres_solve + solvation energy on the resident mesh",
        "energy": (f"treecode (Section 2.5), theta {a.theta}" if a.energy == "treecode" else "direct sum"),
        "l2": "flushed between steps (256 MiB write, outside the timed events)",
    }


def peaks(sm_max_mhz, measured=None):
    """Roofline denominators: the measured HBM copy bandwidth (MEASURED_PEAKS.json) and the
    FP32 / FP64 FMA rates measured by pb_measure_alu_peaks in this run; if the probe did not
    run, FP32 from unit counts (152 SMs x 128 lanes x 2 flops x clock) and FP64 at the part's
    nominal 1.25 TFLOP/s."""
    mhz = sm_max_mhz or 2070.0
    hbm = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm = json.load(f).get("hbm_gbs")
    except OSError:
        pass
    pk = {"fp32_tflops": 152 * 128 * 2 * mhz * 1e6 / 1e12, "fp64_tflops": 1.25, "hbm_gbs": hbm or 6800.0,
          "hbm_source": "measured" if hbm else "fallback", "alu_source": "derived / nominal"}
    if measured:
        pk["fp32_tflops_derived"], pk["fp64_tflops_nominal"] = pk["fp32_tflops"], pk["fp64_tflops"]
        pk["fp32_tflops"], pk["fp64_tflops"] = measured
        pk["alu_source"] = "measured: FMA-chain probe (pb_measure_alu_peaks) in this run"
    return pk


FLOPS_PER_SS_POINT = 100  # FP64 formula count of one Sauter-Schwab point (maps, kernel parts, sums)
# FP32 instructions of one float-float Sauter-Schwab point by class (one shared vertex, a shared
# edge, identical), counted from csrc/singular.cu and csrc/ff.cuh: the primitives cost two-sum 6,
# ff_add 11, ff_mul 7, ff_sqr 7, ff_rsqrt 25, the screening series 122; the six weighted kernel
# parts with their accumulation 409 (245 for the two of identical triangles), plus the point's
# x - y (183 / 129 / 75 by class), r^2 (43) and normal projections (50 / 32 / 0).
FF_INST_PER_SS_POINT = {1: 685, 2: 613, 3: 363}
# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch (summed over the phase's kernels
# for one product / one build), by workload, from the captures summarised in profiles/; None
# where no capture of the current kernel exists
TRAFFIC_BYTES = {
    # profiles/k_singular_ff1_kirkwood_l6.md (singular); the near-field kernel has changed since
    # its sphere capture
    "sphere_l6_p8_leaf64": {"near": None, "m2l": None, "singular": 2.0755e7, "pcbuild": None},
    # profiles/traffic_molecule20k_mixed_p8.md: near, the six MtL levels of one product, the
    # singular pass, the three block-inversion classes of one build
    "molecule_20000_p8_leaf64": {"near": 1.4520e8, "m2l": 7.100e8, "singular": 1.9617e9, "pcbuild": 4.4800e9},
}


def traffic(name, wl_key):
    return TRAFFIC_BYTES.get(wl_key, {}).get(name)


def workload_key(a, N):
    if a.workload == "sphere":
        return f"sphere_l{a.level}_p{a.p}_leaf{a.leaf}"
    return f"molecule_{a.atoms}_p{a.p}_leaf{a.leaf}"


def phase_roofline(name, tv, stats, N, a, prec, pk, wl_key=None):
    """Algorithmic work of one timed launch of a phase over its CUDA-event duration."""
    from math import comb

    from paper_2110_13778_gb300 import pb

    tot_ms, n = tv
    avg_ms = tot_ms / n
    fp32 = prec == pb.PB_MIXED
    if name == "near":
        units = stats["near_pairs"] - N
        flops = units * FLOPS_PER_NEAR_PAIR
        peak = pk["fp32_tflops"] if fp32 else pk["fp64_tflops"]
        work = f"{units} element pairs x {FLOPS_PER_NEAR_PAIR} flops"
    elif name == "m2l":
        pairs = stats["ninter"]
        orders = stats["order"]
        flops = sum(2 * 2 * comb(orders[l] + 6, 6) * pairs[l] for l in range(len(pairs)))
        peak = pk["fp32_tflops"] if fp32 else pk["fp64_tflops"]
        work = f"{sum(pairs)} cluster pairs x 2 kernels x 2 C(p+6,6) flops"
    elif name == "pcbuild":
        # Gauss-Jordan inversion of every block: m^3 FMAs (2 m^3 flops), in the working precision;
        # the assembly (n^2 kernel evaluations per block) is not counted
        flops = 2.0 * stats["pc_sum_m3"]
        if not flops:
            return None
        peak = pk["fp32_tflops"] if fp32 else pk["fp64_tflops"]
        work = f"{stats['pc_blocks']} blocks (m <= {stats['pc_max']}), sum 2 m^3 flops"
    elif name == "singular":
        q4 = 3 ** 4
        cls = stats["touch_class"]
        pts = {3: q4 * 3 * cls[3], 2: q4 * 5 * cls[2] // 2, 1: q4 * 2 * cls[1] // 2}
        points = sum(pts.values())
        if fp32:
            # float-float on the FP32 pipe: FP32 instructions against the FMA issue rate
            inst = sum(FF_INST_PER_SS_POINT[c] * pts[c] for c in pts)
            ach = inst / (avg_ms * 1e-3) / 1e12
            peak = pk["fp32_tflops"] / 2
            # the same work counted as the method's FP64 arithmetic (~100 flops per point) against
            # the FP32 pipe it runs on
            alg = points * FLOPS_PER_SS_POINT / (avg_ms * 1e-3) / 1e12
            return {"kernel": name, "avg_launch_ms": avg_ms, "bound": "alu", "achieved": ach, "peak": peak,
                    "unit": "Tinst/s", "frac": ach / peak, "traffic": traffic(name, wl_key),
                    "work_per_launch": f"{points} quadrature points x float-float FP32 instructions "
                                       f"{FF_INST_PER_SS_POINT} by class = {inst} instructions",
                    "peak_source": "FP32 FMA instructions per second = FP32 FLOP rate / 2 (" + pk["alu_source"] + ")",
                    "algorithmic": {"achieved": alg, "unit": "TFLOP/s", "peak": pk["fp32_tflops"],
                                    "frac": alg / pk["fp32_tflops"],
                                    "work_per_launch": f"{points} quadrature points x {FLOPS_PER_SS_POINT} flops"}}
        flops = points * FLOPS_PER_SS_POINT
        peak = pk["fp64_tflops"]
        work = f"{points} quadrature points x {FLOPS_PER_SS_POINT} FP64 flops"
    else:
        return None
    ach = flops / (avg_ms * 1e-3) / 1e12
    return {"kernel": name, "avg_launch_ms": avg_ms, "bound": "alu", "achieved": ach, "peak": peak,
            "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic(name, wl_key), "work_per_launch": work,
            "peak_source": ("FP32 " if peak == pk["fp32_tflops"] else "FP64 ") + pk["alu_source"]}


def run_ours(a):
    rank, world, local = dist_setup(a.gpus)
    import torch

    torch.cuda.set_device(local)
    from paper_2110_13778_gb300 import build, pb

    build.build()
    mesh = workload(a.level, kind=a.workload, atoms=a.atoms, h=a.grid, clean=not a.raw_mesh)
    N = mesh.nt
    prec = pb.PB_MIXED if a.precision == "mixed" else pb.PB_FP64
    stream = torch.cuda.current_stream().cuda_stream

    def make_ctx(precision):
        prm = pb.params(eps_in=1.0, eps_out=80.0, kappa=0.1257, eta0=a.eta0, leaf_size=a.leaf, p=a.p, qs=3,
                        precision=precision, precond=pb.PB_PRECOND_BLOCK)
        return pb.pb_create(prm, stream)

    ctx = make_ctx(prec)
    pb.pb_mesh_upload(ctx, mesh.verts, mesh.tris, mesh.qpos, mesh.q)
    tuned = None
    if a.autotune:
        # leaf size (32-128) and per-level orders (4, 6, 8) chosen on this mesh, product error
        # <= 1e-4 against order 10; untimed setup, reported in config
        t0 = time.perf_counter()
        tuned = pb.pb_autotune(ctx, tol=1e-4, matvecs_per_solve=9, nrhs=1)
        tuned["seconds"] = time.perf_counter() - t0
        tuned["order"] = tuned["order"][:pb.pb_get_tree_stats(ctx)["levels"] + 1]
    x = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def energy(c):
        if a.energy == "treecode":
            return pb.pb_solvation_energy_treecode(c, x, a.theta)
        return pb.pb_solvation_energy(c, x)

    def step(c):
        pb.pb_build_tree(c)
        info = pb.pb_gmres_solve(c, x, tol=a.tol, max_iter=2000, restart=a.restart)
        return info, energy(c)

    for _ in range(a.warmup):
        step(ctx)
    torch.cuda.synchronize()
    pb.pb_set_timing(ctx, 1)
    n0 = pb.pb_get_launch_count(ctx)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    times, matvecs, iters, energies = [], 0, [], []
    # per-phase event times, read after every step (outside its events: the library keeps the
    # first 256 intervals per phase between reads)
    phases = {}
    barrier(world)
    with ClockSampler(local) as clk:
        for _ in range(a.steps):
            flush.zero_()
            torch.cuda.synchronize()
            ev0.record()
            info, E = step(ctx)
            ev1.record()
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
            matvecs += info.matvecs
            iters.append(info.iterations)
            energies.append(E)
            for k, (t, n) in pb.pb_get_timing(ctx).items():
                t0, n0_ = phases.get(k, (0.0, 0))
                phases[k] = (t0 + t, n0_ + n)
    barrier(world)
    launches = pb.pb_get_launch_count(ctx) - n0
    pb.pb_set_timing(ctx, 0)

    # the same steps with per-phase timing off: each solve is then one CUDA-graph launch with
    # its stopping test on the device (conditional WHILE nodes), no host read per iteration
    g0 = pb.pb_get_graph_launches(ctx)
    dtimes, dmv = [], 0
    for _ in range(a.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ev0.record()
        info_d, E_d = step(ctx)
        ev1.record()
        torch.cuda.synchronize()
        dtimes.append(ev0.elapsed_time(ev1))
        dmv += info_d.matvecs
    device_driven = {"value": world * N * dmv / dist_max(sum(dtimes) / 1e3, world) / 1e6, "unit": UNIT,
                     "ms_per_step": float(np.mean(dtimes)), "graph_launches": pb.pb_get_graph_launches(ctx) - g0,
                     "energy_kcal": E_d}
    stats = pb.pb_get_tree_stats(ctx)
    t_total = sum(times) / 1e3
    t_max = dist_max(t_total, world)
    value = world * N * matvecs / t_max / 1e6

    # the other energy evaluation on the last solution (untimed), for the treecode's error
    E_other = pb.pb_solvation_energy(ctx, x) if a.energy == "treecode" else pb.pb_solvation_energy_treecode(
        ctx, x, a.theta)

    # matrix-vector product alone, resident, L2 warm (reported beside the step metric)
    xv = torch.rand(2 * N, dtype=torch.float64, device="cuda")
    yv = torch.empty_like(xv)
    for _ in range(3):
        pb.pb_matvec(ctx, xv, yv)
    torch.cuda.synchronize()
    ev0.record()
    nmv = 20
    for _ in range(nmv):
        pb.pb_matvec(ctx, xv, yv)
    ev1.record()
    torch.cuda.synchronize()
    t_mv = ev0.elapsed_time(ev1) / nmv

    # the far field alone (nothing beside it on the GPU), per-phase events: the MtL's rate on its
    # own, reported beside its rate inside the step (where it shares the SMs with the near field)
    pb.pb_set_timing(ctx, 1)
    pb.pb_get_timing(ctx)
    for _ in range(10):
        pb.pb_matvec_part(ctx, xv, yv, 2)
    torch.cuda.synchronize()
    far_alone = pb.pb_get_timing(ctx)
    pb.pb_set_timing(ctx, 0)

    # end to end through the public API with host buffers
    pin = lambda arr: torch.from_numpy(np.ascontiguousarray(arr)).pin_memory().numpy()
    hv, ht, hqp, hq = pin(mesh.verts), pin(mesh.tris), pin(mesh.qpos), pin(mesh.q)
    xh = torch.empty(2 * N, dtype=torch.float64).pin_memory()
    e2e_t, e2e_mv = [], 0
    for k in range(a.steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pb.pb_mesh_upload(ctx, hv, ht, hqp, hq)
        info, E = step(ctx)
        xh.copy_(x)
        torch.cuda.synchronize()
        if k > 0:
            e2e_t.append(time.perf_counter() - t0)
            e2e_mv += info.matvecs
    e2e_value = world * N * e2e_mv / dist_max(sum(e2e_t), world) / 1e6
    h2d = hv.nbytes + ht.nbytes + hqp.nbytes + hq.nbytes
    d2h = 2 * N * 8 + 8

    # plain FP64 method on the same box and mesh, for the precision comparison: the same step
    # (build + solve + energy), then as many timed steps as fit the budget (at most --steps).
    # An untimed warm-up step comes first only where a step is short: at a minute or more per
    # FP64 step its one-time costs (pool growth, table upload) are below 1 %
    fp64 = None
    if not a.no_fp64_compare and prec == pb.PB_MIXED:
        c64 = make_ctx(pb.PB_FP64)
        pb.pb_mesh_upload(c64, mesh.verts, mesh.tris, mesh.qpos, mesh.q)
        fp64_warm = t_total / a.steps < 1.0
        if fp64_warm:
            step(c64)
        t64, mv64, it64 = [], 0, []
        while len(t64) < a.steps and (not t64 or sum(t64) / 1e3 + t64[-1] / 1e3 <= a.fp64_budget):
            flush.zero_()
            torch.cuda.synchronize()
            ev0.record()
            info64, E64 = step(c64)
            ev1.record()
            torch.cuda.synchronize()
            t64.append(ev0.elapsed_time(ev1))
            mv64 += info64.matvecs
            it64.append(info64.iterations)
        ms64 = float(np.mean(t64))
        fp64 = {"steps": len(t64), "warmup": int(fp64_warm), "ms_per_step": ms64, "step_ms": t64, "iterations": it64,
                "matvecs_per_step": mv64 / len(t64), "value_melem_s": N * mv64 / (sum(t64) / 1e3) / 1e6,
                "energy_kcal": E64, "rel_energy_diff_mixed_vs_fp64": abs(energies[-1] - E64) / abs(E64),
                "solve_time_ratio_fp64_over_mixed": ms64 / (1e3 * t_total / a.steps)}
        pb.pb_destroy(c64)
    pb.pb_destroy(ctx)

    clocks = clk.summary()
    try:
        measured = pb.pb_measure_alu_peaks(torch.cuda.current_stream().cuda_stream)
    except pb.PBError:
        measured = None
    pk = peaks(clocks.get("sm_max_mhz"), measured)
    per_step = {k: v[0] / a.steps for k, v in phases.items()}
    # roofline of the product's dominant kernel, the near field (and of the other hot
    # kernels, for the report)
    kernels = {k: v for k, v in phases.items() if v[1] > 0}
    wl_key = workload_key(a, N)
    rooflines = {k: phase_roofline(k, kernels[k], stats, N, a, prec, pk, wl_key)
                 for k in ("near", "m2l", "singular", "pcbuild") if k in kernels}
    if tuned:  # the ncu traffic figures were taken at the default leaf size and order
        for r in rooflines.values():
            if r:
                r["traffic"] = None
    if far_alone.get("m2l", (0, 0))[1] > 0:
        iso = phase_roofline("m2l", far_alone["m2l"], stats, N, a, prec, pk, wl_key)
        if iso:
            iso["note"] = "far field alone (pb_matvec_part, which = 2): no near field beside it"
            rooflines["m2l_alone"] = iso
    roof = rooflines.get("near")

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        v, nrows, dt = cpu_oracle_rate(mesh, budget_s=20.0)
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{nrows} dense Galerkin rows of A x of the {N}-triangle workload ({dt:.1f} s)"}
    if rank == 0:
        Ek = None
        if a.workload == "sphere":
            from oracle import kirkwood

            Ek = kirkwood.series(mesh.qpos, mesh.q, 20.0, 1.0, 80.0, 0.1257)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * t_max / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if prec == pb.PB_MIXED else "f64", "data": "synthetic",
            "config": dict(config_dict(a, mesh), **({"autotune": {
                "leaf_size": tuned["leaf_size"], "order_per_level": tuned["order"], "rel_err": tuned["rel_err"],
                "seconds": tuned["seconds"], "untimed": True}} if tuned else {})), "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
            "gmres_iterations": iters, "matvecs_per_step": matvecs / a.steps,
            "phases_ms_per_step": per_step, "phase_rooflines": rooflines, "matvec_ms": t_mv, "matvec_only_melem_s": N / t_mv / 1e3,
            "energy_kcal": energies[-1], ("energy_direct_kcal" if a.energy == "treecode" else "energy_treecode_kcal"):
            E_other, "kirkwood_series_kcal": Ek, "tree": stats, "fp64_method": fp64,
            "device_driven_gmres": device_driven,
            "peaks": pk,
        }
        print(json.dumps(line))
    return 0


def batch_sizes(rank, molecules, max_atoms):
    """Each rank's own molecules (weak scaling: the ranks share no data): atom counts
    log-uniform in [200, max_atoms] from a rank-seeded generator, which also draws the states."""
    rng = np.random.default_rng(4000 + rank)
    return rng, np.exp(rng.uniform(np.log(200), np.log(max_atoms), size=molecules)).astype(int)


def run_batch(a):
    """Many protein-like molecules of uneven size, each with `states` charge states (5 % of the
    charges flipped per state), all solved in one CUDA-graph launch (pb_batch_solve_states: one
    branch per molecule, every GMRES stopping on the device). One step = every molecule's
    pb_build_tree + the one batched solve (energies included). value = sum over molecules and
    states of N x matvecs / step time."""
    rank, world, local = dist_setup(a.gpus)
    import torch

    torch.cuda.set_device(local)
    from paper_2110_13778_gb300 import build, molecules, pb

    build.build()
    rng, sizes = batch_sizes(rank, a.molecules, a.max_atoms)
    t0 = time.perf_counter()
    mols = [molecules.molecule(int(n), 5000 + 97 * rank + k, a.grid, clean=not a.raw_mesh)[0]
            for k, n in enumerate(sizes)]
    t_gen = time.perf_counter() - t0
    states = []
    for m in mols:
        Q = np.repeat(m.q[None, :], a.states, axis=0)
        for s_ in range(1, a.states):
            flip = rng.random(m.q.size) < 0.05
            Q[s_, flip] = -Q[s_, flip]
        states.append(Q)
    stream = torch.cuda.current_stream().cuda_stream
    prm = pb.params(eps_in=1.0, eps_out=80.0, kappa=0.1257, eta0=a.eta0, leaf_size=a.leaf, p=a.p, qs=3,
                    precision=pb.PB_MIXED if a.precision == "mixed" else pb.PB_FP64, precond=pb.PB_PRECOND_BLOCK)
    # one context per molecule, its leaf size and order chosen by the autotuner (untimed)
    ctxs, tuned = [], []
    t0 = time.perf_counter()
    for m in mols:
        cx = pb.pb_create(prm, stream)
        pb.pb_mesh_upload(cx, m.verts, m.tris, m.qpos, m.q)
        if not a.no_autotune:
            r = pb.pb_autotune(cx, tol=1e-4, matvecs_per_solve=10, nrhs=a.states)
            r["order"] = r["order"][:pb.pb_get_tree_stats(cx)["levels"] + 1]
            tuned.append(r)
        ctxs.append(cx)
    t_tune = time.perf_counter() - t0
    Xs = [torch.empty((a.states, 2 * m.nt), dtype=torch.float64, device="cuda") for m in mols]
    restart = a.batch_restart

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    split = {"build_ms": [], "solve_ms": []}

    def step():
        ev[0].record()
        for cx in ctxs:
            pb.pb_build_tree(cx)
        ev[1].record()
        E, infos = pb.pb_batch_solve_states(ctxs, states, Xs, tol=a.tol, max_iter=500, restart=restart)
        ev[2].record()
        torch.cuda.synchronize()
        split["build_ms"].append(ev[0].elapsed_time(ev[1]))
        split["solve_ms"].append(ev[1].elapsed_time(ev[2]))
        return sum(i.matvecs * m.nt for inf, m in zip(infos, mols) for i in inf), E, infos

    for _ in range(a.warmup):
        step()
    split["build_ms"].clear()
    split["solve_ms"].clear()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    n0 = sum(pb.pb_get_launch_count(cx) for cx in ctxs)
    g0 = [pb.pb_get_graph_launches(cx) for cx in ctxs]
    barrier(world)
    units, times = 0, []
    with ClockSampler(local) as clk:
        for _ in range(a.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            u, E, infos = step()
            units += u
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    barrier(world)
    dt = dist_max(sum(times), world)
    launches = sum(pb.pb_get_launch_count(cx) for cx in ctxs) - n0
    graph_launches = [pb.pb_get_graph_launches(cx) - g for cx, g in zip(ctxs, g0)]
    # the same solves one molecule at a time (pb_solve_states, batched states per molecule, two
    # graph launches each), for the energies' agreement and the gain of the single launch
    torch.cuda.synchronize()
    ev[0].record()
    worst = 0.0
    seq_units = 0
    for k, (cx, m) in enumerate(zip(ctxs, mols)):
        Xr = torch.empty_like(Xs[k])
        Er, ir = pb.pb_solve_states(cx, states[k], Xr, tol=a.tol, max_iter=500, restart=restart, warm=2)
        worst = max(worst, float(np.max(np.abs(Er - E[k]) / np.abs(Er))))
        seq_units += sum(i.matvecs * m.nt for i in ir)
    ev[1].record()
    torch.cuda.synchronize()
    t_seq = ev[0].elapsed_time(ev[1]) / 1e3
    mem = torch.cuda.mem_get_info()
    for cx in ctxs:
        pb.pb_destroy(cx)
    if rank == 0:
        print(json.dumps({
            "metric": "batched molecules x charge states: element-matvecs per second (builds + one-launch solve)",
            "value": world * units / dt / 1e6, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if a.precision == "mixed" else "f64", "data": "synthetic",
            "clocks": clk.summary(), "gpu_launches": launches, "graph_launches_per_step": [g / a.steps for g in graph_launches],
            "iterations_max": max(i.iterations for inf in infos for i in inf),
            "build_ms_per_step": float(np.mean(split["build_ms"])), "solve_ms_per_step": float(np.mean(split["solve_ms"])),
            "one_by_one": {"solve_ms": 1e3 * t_seq, "value_solves_only": seq_units / t_seq / 1e6,
                           "batch_value_solves_only": units / a.steps / (np.mean(split["solve_ms"]) / 1e3) / 1e6,
                           "max_rel_energy_diff_vs_batch": worst},
            "device_memory_free_gb": mem[0] / 1e9, "device_memory_total_gb": mem[1] / 1e9,
            "config": {"workload": f"{a.molecules} protein-like molecules, atoms log-uniform in [200, {a.max_atoms}] "
                                   f"({int(sum(sizes))} atoms, {sum(m.nt for m in mols)} triangles in all; largest "
                                   f"{max(m.nt for m in mols)}) x {a.states} charge states (5 % of charges flipped)",
                       "atoms": [int(n) for n in sizes], "triangles": [m.nt for m in mols],
                       "eta0": a.eta0, "restart": restart, "host_generation_s": t_gen,
                       "l2": "flushed (256 MiB write) before each step, outside the timed events",
                       "autotune": ({"leaf_size": [t["leaf_size"] for t in tuned], "p": [t["p"] for t in tuned],
                                     "order_per_level": [t["order"] for t in tuned],
                                     "rel_err": [t["rel_err"] for t in tuned], "seconds": t_tune}
                                    if tuned else {"leaf_size": a.leaf, "p": a.p})}}))
    return 0


def run_precond(a):
    """Diagonal against block-diagonal preconditioning (Section 2.6; the paper's Table 4 on
    synthetic protein-like surfaces instead of its 27 proteins): for molecules of 500 to 4000
    atoms, GMRES iterations and times (build, solve) with no preconditioner, the 2 x 2 diagonal
    blocks ("d") and leaf blocks cut to at most 16, 32, 64 and 96 elements ("bd"; smaller blocks
    stand for designated levels below the leaves). Mixed precision, p = 8, GMRES to 1e-6."""
    rank, world, local = dist_setup(a.gpus)
    import torch

    torch.cuda.set_device(local)
    from paper_2110_13778_gb300 import build, molecules, pb

    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    forms = [("none", pb.PB_PRECOND_NONE, 0), ("d", pb.PB_PRECOND_DIAG, 0)] + \
            [(f"bd{b}", pb.PB_PRECOND_BLOCK, b) for b in (16, 32, 64, 96)]
    rows = []
    clk = ClockSampler(local)
    clk.__enter__()
    from math import isfinite

    for atoms, clean in ((500, False), (1000, False), (2000, False), (4000, False), (500, True), (1000, True),
                         (2000, True), (4000, True), (8000, True)):
        m = molecules.molecule(atoms, 7000 + atoms, a.grid, clean=clean)[0]
        row = {"atoms": atoms, "N": m.nt, "mesh": "short edges collapsed" if clean else "raw marching tetrahedra"}
        for name, pc, b in forms:
            prm = pb.params(eps_in=1.0, eps_out=80.0, kappa=0.1257, eta0=a.eta0, leaf_size=a.leaf, p=a.p, qs=3,
                            precision=pb.PB_MIXED, precond=pc, pc_block=b)
            cx = pb.pb_create(prm, stream)
            pb.pb_mesh_upload(cx, m.verts, m.tris, m.qpos, m.q)
            x = torch.zeros(2 * m.nt, dtype=torch.float64, device="cuda")
            bt, st = [], []
            for it in range(a.warmup + a.steps):
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                torch.cuda.synchronize()
                e0.record()
                pb.pb_build_tree(cx)
                e1.record()
                info = pb.pb_gmres_solve(cx, x, tol=a.tol, max_iter=1000, restart=50, raise_on_fail=False)
                e2.record()
                torch.cuda.synchronize()
                if it >= a.warmup:
                    bt.append(e0.elapsed_time(e1))
                    st.append(e1.elapsed_time(e2))
            E = pb.pb_solvation_energy(cx, x)
            ts = pb.pb_get_tree_stats(cx)
            pb.pb_destroy(cx)
            row[name] = {"iterations": info.iterations, "status": info.status, "build_ms": statistics.median(bt),
                         "solve_ms": statistics.median(st), "total_ms": statistics.median(bt) + statistics.median(st),
                         "energy_kcal": E if isfinite(E) else None, "blocks": ts["pc_blocks"], "max_block": ts["pc_max"]}
        rows.append(row)
    clk.__exit__(None, None, None)
    if rank != 0:
        return 0
    print(json.dumps({
        "metric": "GMRES iterations and time to 1e-6: diagonal vs block-diagonal preconditioner", "value":
        float(np.mean([r["d"]["iterations"] / r["bd96"]["iterations"] for r in rows])), "unit": "iterations d / bd (mean)",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "clocks": clk.summary(), "rows": rows,
        "config": {"workload": "protein-like molecules of 500-8000 atoms, marching tetrahedra on a "
                               f"{a.grid} A grid: raw (narrow and tiny triangles included) and with edges shorter "
                               f"than {a.grid / 10:.2f} A collapsed", "p": a.p, "eta0": a.eta0,
                   "leaf_size": a.leaf}}))
    return 0


def run_linear(a):
    """The piecewise-linear basis (continuous hat functions, Section 2.3) on a protein-like
    molecule: one step = pb_build_tree + pb_gmres_solve + the solvation energy, vertex unknowns,
    order-2 regular rule (4 points per element), p = 8, mixed precision, the 2 x 2 vertex-block
    preconditioner; value = N_elements x products / step time (the default metric's unit). The
    piecewise-constant step on the same molecule and rule is timed beside it. Roofline: the
    near field k_near_p1, 16 point pairs per near element pair x 75 flops."""
    rank, world, local = dist_setup(a.gpus)
    import torch

    torch.cuda.set_device(local)
    from paper_2110_13778_gb300 import build, pb

    build.build()
    mesh = workload(kind="molecule", atoms=a.atoms, h=a.grid, clean=not a.raw_mesh)
    N, nv = mesh.nt, mesh.verts.shape[0]
    prec = pb.PB_MIXED if a.precision == "mixed" else pb.PB_FP64
    stream = torch.cuda.current_stream().cuda_stream
    qr = 2
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def arm(basis):
        prm = pb.params(eps_in=1.0, eps_out=80.0, kappa=0.1257, eta0=a.eta0, leaf_size=a.leaf, p=a.p, qs=3,
                        precision=prec, precond=pb.PB_PRECOND_BLOCK, qr=qr, basis=basis)
        cx = pb.pb_create(prm, stream)
        pb.pb_mesh_upload(cx, mesh.verts, mesh.tris, mesh.qpos, mesh.q)
        n = 2 * (nv if basis == pb.PB_BASIS_LINEAR else N)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")

        def step():
            pb.pb_build_tree(cx)
            info = pb.pb_gmres_solve(cx, x, tol=a.tol, max_iter=2000, restart=a.restart)
            return info, pb.pb_solvation_energy(cx, x)

        for _ in range(a.warmup):
            step()
        torch.cuda.synchronize()
        pb.pb_set_timing(cx, 1)
        n0 = pb.pb_get_launch_count(cx)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times, mv, its = [], 0, []
        phases = {}
        for _ in range(a.steps):
            flush.zero_()
            torch.cuda.synchronize()
            ev0.record()
            info, E = step()
            ev1.record()
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1))
            mv += info.matvecs
            its.append(info.iterations)
            for k, (t, n) in pb.pb_get_timing(cx).items():
                t0, n0_ = phases.get(k, (0.0, 0))
                phases[k] = (t0 + t, n0_ + n)
        launches = pb.pb_get_launch_count(cx) - n0
        pb.pb_set_timing(cx, 0)
        stats = pb.pb_get_tree_stats(cx)
        pb.pb_destroy(cx)
        return {"times": times, "matvecs": mv, "iterations": its, "energy": E, "phases": phases, "launches": launches,
                "stats": stats}

    with ClockSampler(local) as clk:
        lin = arm(pb.PB_BASIS_LINEAR)
    const = arm(pb.PB_BASIS_CONSTANT)
    t_max = dist_max(sum(lin["times"]) / 1e3, world)
    value = world * N * lin["matvecs"] / t_max / 1e6
    pk = peaks(clk.summary().get("sm_max_mhz"), pb.pb_measure_alu_peaks(stream))
    near_ms, near_n = lin["phases"]["near"]
    avg = near_ms / max(near_n, 1)
    pairs = lin["stats"]["near_pairs"] - N  # the identical pair is stored whole with the touching blocks
    flops = pairs * (qr * qr) ** 2 * FLOPS_PER_NEAR_PAIR
    peak = pk["fp32_tflops"] if prec == pb.PB_MIXED else pk["fp64_tflops"]
    ach = flops / (avg * 1e-3) / 1e12
    # the weighted Sauter-Schwab pass (FP64, once per build): per cube point and sub-map the
    # point's kernel parts (FLOPS_PER_SS_POINT) plus 9 weight products and 54 weighted FMAs;
    # 2 / 5 / 6 sub-maps for unordered pairs sharing a vertex / an edge / identical
    tc = lin["stats"]["touch_class"]
    sub = tc[1] // 2 * 2 + tc[2] // 2 * 5 + N * 6
    sflops = 3 ** 4 * sub * (FLOPS_PER_SS_POINT + 9 + 2 * 54)
    s_ms, s_n = lin["phases"]["singular"]
    s_avg = s_ms / max(s_n, 1)
    s_ach = sflops / (s_avg * 1e-3) / 1e12
    sing = {"kernel": "k_singular_p1", "avg_launch_ms": s_avg, "bound": "alu", "achieved": s_ach,
            "peak": pk["fp64_tflops"], "unit": "TFLOP/s", "frac": s_ach / pk["fp64_tflops"], "traffic": None,
            "work_per_launch": f"81 cube points x {sub} sub-map evaluations x {FLOPS_PER_SS_POINT + 9 + 2 * 54} FP64 flops",
            "peak_source": "FP64 " + pk["alu_source"]}
    if rank != 0:
        return 0
    print(json.dumps({
        "metric": "piecewise-linear FMM matvec Melem/s (whole solve: setup + GMRES to 1e-6 + energy)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": float(np.mean(lin["times"])), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == pb.PB_MIXED else "f64", "data": "synthetic", "clocks": clk.summary(),
        "gpu_launches": lin["launches"], "gmres_iterations": lin["iterations"],
        "matvecs_per_step": lin["matvecs"] / a.steps, "energy_kcal": lin["energy"],
        "phases_ms_per_step": {k: v[0] / a.steps for k, v in lin["phases"].items() if v[1]},
        "roofline": {"kernel": "near (k_near_tile<4> on the rule's points)" if prec == pb.PB_MIXED else "near (k_near_p1)",
                     "avg_launch_ms": avg, "bound": "alu", "achieved": ach, "peak": peak,
                     "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                     "work_per_launch": f"{pairs} element pairs x {(qr * qr) ** 2} point pairs x "
                                        f"{FLOPS_PER_NEAR_PAIR} flops",
                     "peak_source": pk["alu_source"]},
        "phase_rooflines": {"singular_p1": sing},
        "piecewise_constant": {"ms_per_step": float(np.mean(const["times"])), "gmres_iterations": const["iterations"],
                               "energy_kcal": const["energy"],
                               "value": world * N * const["matvecs"] / dist_max(sum(const["times"]) / 1e3, world)
                               / 1e6},
        "config": {"workload": f"protein-like molecule: {a.atoms}-atom self-avoiding walk, Gaussian isosurface at 1.0 "
                               f"on a {a.grid} A grid, {N} triangles, {nv} vertices, {mesh.nc} charges",
                   "basis": "continuous piecewise-linear (hat functions at the vertices)", "qr": qr, "p": a.p,
                   "eta0": a.eta0, "leaf_size": a.leaf, "precision": a.precision,
                   "precond": "2 x 2 vertex blocks of the exact diagonal",
                   "gmres": f"GMRES({a.restart}) tol {a.tol}",
                   "l2": "flushed between steps (256 MiB write, outside the timed events)"}}))
    return 0


def run_learned(a):
    """Learned warm start against a zero start, and both against plain FP64 from zero.

    Training (untimed): `train-molecules` protein-like molecules of `train-atoms` atoms (default
    50-500, log-uniform),
    each solved from zero by the mixed-precision solver; the network (18 -> 128 -> 128 -> 128
    -> 2, BF16 tensor-core kernels) is fitted to their scaled solutions by Adam. Evaluation:
    the `atoms`-atom molecule, three arms per step, each pb_build_tree + solve to `tol` +
    energy: mixed precision from the learned start (network inference included), mixed from
    zero, FP64 from zero. value = the learned arm's time per solve."""
    rank, world, local = dist_setup(a.gpus)
    import torch

    torch.cuda.set_device(local)
    from paper_2110_13778_gb300 import build, molecules, pb, warmstart

    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(6000 + rank)
    counts = np.exp(rng.uniform(np.log(a.train_atoms[0]), np.log(a.train_atoms[1]), a.train_molecules)).astype(int)
    t0 = time.perf_counter()
    F, T = warmstart.make_dataset(counts, seed=6100 + rank, grid=a.grid, clean=not a.raw_mesh)
    t_data = time.perf_counter() - t0
    net = pb.pb_mlp_create(pb.NFEAT, warmstart.WIDTH, warmstart.DEPTH, 2, seed=17, stream=stream)
    first, last, t_train = warmstart.train(net, F, T, steps=a.train_steps, batch=8192, lr=1e-3, lr_final=1e-4)
    mesh = workload(kind="molecule", atoms=a.atoms, h=a.grid, clean=not a.raw_mesh)
    N = mesh.nt

    def prm(precision):
        return pb.params(eps_in=1.0, eps_out=80.0, kappa=0.1257, eta0=a.eta0, leaf_size=a.leaf, p=a.p, qs=3,
                         precision=precision, precond=pb.PB_PRECOND_BLOCK)

    arms = {"learned_mixed": (pb.PB_MIXED, True), "zero_mixed": (pb.PB_MIXED, False), "zero_fp64": (pb.PB_FP64, False)}
    ctxs = {}
    for k, (precision, _) in arms.items():
        ctxs[k] = pb.pb_create(prm(precision), stream)
        pb.pb_mesh_upload(ctxs[k], mesh.verts, mesh.tris, mesh.qpos, mesh.q)
    x = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    res = {k: {"ms": [], "info": None, "E": None} for k in arms}

    def run(k):
        precision, learned = arms[k]
        c = ctxs[k]
        pb.pb_build_tree(c)
        if learned:
            pb.pb_learned_guess(c, net, x)
        else:
            x.zero_()
        info = pb.pb_gmres_solve(c, x, tol=a.tol, max_iter=2000, restart=a.restart, use_x0=learned)
        return info, pb.pb_solvation_energy(c, x)

    clk = ClockSampler(local)
    for it in range(a.warmup + a.steps):
        if it == a.warmup:
            clk.__enter__()
        for k in arms:
            flush.fill_(it & 255)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            info, E = run(k)
            e1.record()
            torch.cuda.synchronize()
            if it >= a.warmup:
                res[k]["ms"].append(e0.elapsed_time(e1))
                res[k]["info"], res[k]["E"] = info, E
    clk.__exit__(None, None, None)
    for c in ctxs.values():
        pb.pb_destroy(c)
    pb.pb_mlp_destroy(net)
    if rank != 0:
        return 0
    ms = {k: statistics.median(v["ms"]) for k, v in res.items()}
    Eref = res["zero_fp64"]["E"]
    arms_out = {k: {"ms": ms[k], "iterations": v["info"].iterations, "matvecs": v["info"].matvecs,
                    "initial_residual": v["info"].initial_residual, "rel_residual": v["info"].rel_residual,
                    "energy_kcal": v["E"], "energy_rel_err_vs_fp64": abs(v["E"] - Eref) / abs(Eref)}
                for k, v in res.items()}
    print(json.dumps({
        "metric": "PB solve time to 1e-6 residual (build + solve + energy), learned+mixed", "value": ms["learned_mixed"],
        "unit": "ms", "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": sum(ms.values()),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64+bf16",
        "data": "synthetic", "clocks": clk.summary(), "arms": arms_out,
        "speedup_vs_fp64_zero": ms["zero_fp64"] / ms["learned_mixed"],
        "speedup_vs_mixed_zero": ms["zero_mixed"] / ms["learned_mixed"],
        "training": {"molecules": int(a.train_molecules), "atoms": [int(c) for c in counts], "rows": int(F.shape[0]),
                     "data_seconds": t_data, "steps": a.train_steps, "train_seconds": t_train,
                     "loss_first": first, "loss_last": last},
        "config": {"workload": f"protein-like molecule, {a.atoms} atoms, grid {a.grid} A, {N} triangles" +
                               ("" if a.raw_mesh else " (short edges collapsed)"),
                   "p": a.p, "eta0": a.eta0, "leaf_size": a.leaf, "gmres": f"GMRES({a.restart}) tol {a.tol}",
                   "l2": "flushed (256 MiB write) before each arm"}}))
    return 0


def main():
    a = args_parse()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "batch":
        return run_batch(a)
    if a.workload == "learned":
        return run_learned(a)
    if a.workload == "precond":
        return run_precond(a)
    if a.workload == "linear":
        return run_linear(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
