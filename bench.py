#!/usr/bin/env python
"""Benchmark of the HHG P1 multigrid V-cycle on one GB300 (per process).

Workload (default): P1 Poisson on the straight-edged annulus r in [0.55, 1],
32 angular x 2 radial quads cut into 128 macro-triangles, refined to level 10
(1025 lattice points per macro-edge, 67.1 M free unknowns), homogeneous
Dirichlet conditions on both circles, b uniform in [-1, 1) from SplitMix64
(seed 1234), FP64.  One step = one V(3,3) cycle (3-colour Gauss-Seidel, full
weighting, linear prolongation, CG on level 0) plus the FP64 residual and its
norm (the solver's convergence test), all on the device.

Printed (one JSON line, rank 0): GDoF/s per V-cycle = free DoFs x cycles /
seconds / 1e9 over all ranks (independent replicas, weak scaling), with
  e2e          the same through the public API from pinned host memory
               (b copied host->device each step, norm read back);
  roofline     the dominant kernel (face Gauss-Seidel) timed by CUDA events
               inside the timed region, against the FP64 ALU peak;
  cpu_baseline the FP64 oracle timed on the host cores on a bounded sample;
  time_to_tol  wall time to a 1e-10 relative FP64 residual: FP64 V-cycles,
               FP32 V-cycles inside FP64 iterative refinement,
               V-cycle-preconditioned conjugate gradients (FP64), and
               flexible CG preconditioned by an FP32 V-cycle.
``--impl reference`` times the oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GDoF/s per V-cycle & time to 1e-10 FP64 residual: mixed/learned vs FP64 (1 GB300)"
UNIT = "GDoF/s"
FP64_OPS_PER_CLK_SM = 2           # FP64 add/mul/fma per clock per SM (cross-checked by the DGEMM probe)
# dram__bytes_read.sum + dram__bytes_write.sum of one level-9 launch of the
# FP64 face sweep (annulus, 128 faces), per (kernel variant, split), from the
# ncu captures summarised under profiles/; None until captured
TRAFFIC_L9 = {(1, 32): 391.016448e6 + 113.307136e6}   # k_gs_sweep<double, 0, 0, 1, 1, 0>, default split


# ------------------------------------------------------------------ ranks
def rank_barrier(world):
    """Barrier over the ranks of the job (one process per GPU)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def rank_max(v, world, device):
    """The maximum of a per-rank value over all ranks (the slowest rank's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, steps, ms):
    """Whole-job throughput (weak scaling: every rank processes its own
    replica): all ranks' units per second, in units of 1e9."""
    return world * units_per_rank * steps / (ms / 1e3) / 1e9


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--level", type=int, default=10)
    ap.add_argument("--cpu-level", type=int, default=8, help="level of the oracle's bounded sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-vark", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-p2", action="store_true")
    ap.add_argument("--no-stokes", action="store_true")
    ap.add_argument("--learned-pairs", type=int, default=10000)
    ap.add_argument("--learned-epochs", type=int, default=12)
    ap.add_argument("--batch-size", type=int, default=64)
    ap.add_argument("--case", default="bench", choices=["bench", "sweep", "cnn", "stokes"],
                    help="sweep: only four forward Gauss-Seidel sweeps on --level in --prec; "
                         "cnn: only --steps applications of the learned smoother's network on "
                         "--level of the variable-coefficient annulus, timed (the small cases of "
                         "the ncu captures under profiles/), no JSON line; stokes: --warmup and --steps "
                         "Uzawa steps on --level of the 256-face annulus, no JSON line")
    ap.add_argument("--prec", default="f64", choices=["f64", "f32"])
    ap.add_argument("--arith", default="ieee", choices=["ieee", "dfloat"],
                    help="arithmetic of the FP64 face kernels in the sweep case")
    return ap.parse_args()


def workload(level):
    from paper_1805_10167_gb300 import inputs
    xy, tri = inputs.annulus_mesh(32, 2)
    return xy, tri, f"annulus-32x2-128faces-L{level}-P1-Poisson-fp64-V(3,3)"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ oracle timing
def oracle_rate(level, cycles, warmup=0):
    """The FP64 oracle (as it stands) on the same annulus at a lower level:
    returns (GDoF/s, seconds per cycle, free DoFs)."""
    from oracle import mesh as om
    from oracle import multigrid as mg
    from paper_1805_10167_gb300 import inputs
    xy, tri = inputs.annulus_mesh(32, 2)
    H = mg.Hierarchy(om.MacroMesh(xy, tri), level)
    lv = H.levels[level]
    b = inputs.uniform_pm1(lv.n, 1234)
    x = np.zeros(lv.n)
    for l in range(1, level + 1):          # assemble the smoother sets and transfers once
        H.sets(l)
        H.P(l)
    for _ in range(warmup):
        mg.vcycle(H, level, x, b, 3, 3)
    t0 = time.perf_counter()
    for _ in range(cycles):
        mg.vcycle(H, level, x, b, 3, 3)
        r = H.residual(level, x, b)
        mg.norm_free(H, level, r)
    dt = time.perf_counter() - t0
    n_free = int(lv.free.sum())
    return n_free * cycles / dt / 1e9, dt / cycles, n_free


def _oracle_worker(q, go, level, cycles, warmup):
    """One process of the all-core oracle baseline: the oracle as it stands
    (single-threaded numpy/scipy) on its own replica of the sample."""
    from oracle import mesh as om
    from oracle import multigrid as mg
    from paper_1805_10167_gb300 import inputs
    xy, tri = inputs.annulus_mesh(32, 2)
    H = mg.Hierarchy(om.MacroMesh(xy, tri), level)
    lv = H.levels[level]
    b = inputs.uniform_pm1(lv.n, 1234)
    x = np.zeros(lv.n)
    for l in range(1, level + 1):
        H.sets(l)
        H.P(l)
    for _ in range(max(1, warmup)):
        mg.vcycle(H, level, x, b, 3, 3)
    q.put(("ready", 0.0, 0.0, 0))
    go.wait()
    t0 = time.time()
    for _ in range(cycles):
        mg.vcycle(H, level, x, b, 3, 3)
        mg.norm_free(H, level, H.residual(level, x, b))
    q.put(("done", t0, time.time(), int(lv.free.sum())))


def oracle_pool_rate(level, cycles, procs=None, warmup=1):
    """The oracle on every host core: `procs` independent replicas (one
    single-threaded process each, started with spawn), released together;
    returns (aggregate GDoF/s, processes, seconds per cycle of one process).
    The oracle solves one problem in one thread, so all cores serve
    independent problems."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    q, go = ctx.Queue(), ctx.Event()
    ps = [ctx.Process(target=_oracle_worker, args=(q, go, level, cycles, warmup)) for _ in range(procs)]
    try:
        for pr in ps:
            pr.start()
        for _ in range(procs):
            q.get(timeout=600)
        go.set()
        res = [q.get(timeout=1200) for _ in range(procs)]
    finally:
        for pr in ps:
            pr.join(timeout=60)
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    t0, t1 = min(r[1] for r in res), max(r[2] for r in res)
    units = sum(r[3] * cycles for r in res)
    per_cycle = float(np.mean([(r[2] - r[1]) / cycles for r in res]))
    return units / (t1 - t0) / 1e9, procs, per_cycle


def fp64_dgemm_probe(dev, n=4096, reps=5):
    """Measured FP64 rate of the device: cuBLAS DGEMM (torch.matmul in
    float64) on n x n operands, CUDA-event timed after warm-up.  A DGEMM runs
    on the FP64 FMA units, so half its FLOP/s is the FP64 instruction rate
    the stencil kernels are held against."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    for _ in range(2):
        torch.matmul(a, b)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        torch.matmul(a, b)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    tflops = 2.0 * n ** 3 / (ms / 1e3) / 1e12
    return {"dgemm_tflops": tflops, "fp64_instr_g_per_s": tflops * 1e3 / 2.0, "n": n, "ms": ms}


def run_batch(args, dev, st):
    """Batch of independent problems (random square triangulations, 2-64
    faces, levels 6-9, b uniform from seed 1000 + k): one merged launch per
    phase and level group, graph-replayed FP32-in-FP64 iterations, autotuned
    face sweeps -- against the same problems solved one after another; and
    the batched flexible CG with an FP32 V-cycle preconditioner."""
    import torch

    from paper_1805_10167_gb300 import hhg, inputs
    probs = inputs.batch_workload(args.batch_size)
    B = hhg.Batch([(xy, tri) for xy, tri, L in probs], [L for xy, tri, L in probs])
    B.tune(stream=st)
    n = len(probs)
    infos = [B.info(p) for p in range(n)]
    bs = [torch.tensor(inputs.uniform_pm1(I.n_nodes, 1000 + p), dtype=torch.float64, device=dev)
          for p, I in enumerate(infos)]
    xs = [torch.zeros_like(b) for b in bs]

    def timed_batch(mode):
        for x in xs:
            x.zero_()
        B.solve(xs, bs, mode=mode, stream=st)           # warm-up (captures the graph)
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, reps = B.solve(xs, bs, mode=mode, stream=st)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, reps
    t_cg, reps_cg = timed_batch(hhg.SOLVE_FPCG)
    t_batch, reps = timed_batch(hhg.SOLVE_IR)
    outer = max(r["iterations"] for r in reps)
    free = sum(I.n_free for I in infos)
    # a level group iterates until its last problem meets the tolerance
    group_its = {}
    for (_, _, L), r in zip(probs, reps):
        group_its[L] = max(group_its.get(L, 0), r["iterations"])
    dof_cycles = sum(I.n_free * group_its[L] for I, (_, _, L) in zip(infos, probs))
    # the same problems one by one through hhg_solve (IR), one mesh each
    t_seq = 0.0
    for p, (xy, tri, L) in enumerate(probs):
        g = hhg.Mesh(xy, tri, L)
        I = g.info(L)
        bi = torch.zeros(I.vec_len, dtype=torch.float64, device=dev)
        xi = torch.zeros_like(bi)
        g.from_canonical(L, bs[p], bi, stream=st)
        g.solve(L, xi, bi, mode=hhg.SOLVE_IR, stream=st)     # warm-up
        xi.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        g.solve(L, xi, bi, mode=hhg.SOLVE_IR, stream=st)
        torch.cuda.synchronize()
        t_seq += time.perf_counter() - t1
        g.close()
    B.close()
    return {"problems": n, "faces": [int(t.shape[0]) for _, t, _ in probs],
            "levels": [int(L) for _, _, L in probs], "free_dofs": int(free),
            "outer_iterations": outer, "group_iterations": {str(k): v for k, v in sorted(group_its.items())},
            "seconds_to_tol": t_batch,
            "gdofs_per_cycle": dof_cycles / t_batch / 1e9,
            "sequential_seconds_to_tol": t_seq, "speedup_vs_sequential": t_seq / t_batch,
            "all_converged": all(r["r_final"] <= 1e-10 * r["r0"] for r in reps),
            "flexible_cg": {"seconds_to_tol": t_cg, "steps": max(r["iterations"] for r in reps_cg),
                            "all_converged": all(r["r_final"] <= 1e-10 * r["r0"] for r in reps_cg),
                            "speedup_vs_batched_ir": t_batch / t_cg}}


def run_p2(args, g, info, b, dev, st, hbm_peak, n_sm, sm_mhz):
    """P2 elements on level L - 1 of the same annulus: their unknowns are the
    level-L lattice (the same 67.1 M free unknowns at L = 10), b the same
    right-hand side.  Time to a 1e-10 relative residual by p-multigrid
    (V(2,2) P2 Gauss-Seidel, a P1 V(3,3) coarse correction on level L - 1)
    and the P2 operator's roofline (FP64 instructions per point: 13 at
    micro-vertex points, 7 at edge points)."""
    import torch
    from paper_1805_10167_gb300 import hhg
    L = args.level
    Lp = L - 1
    x = torch.zeros_like(b)
    g.p2_solve(Lp, x, b, stream=st)             # warm-up (colour tables, graph capture)
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, rep = g.p2_solve(Lp, x, b, stream=st)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    y = torch.zeros_like(b)
    for _ in range(3):
        g.p2_apply(Lp, x, y, stream=st)
    reps = 10
    hhg.profile_begin((1 << hhg.K_FACE_ROWS) | (1 << hhg.K_EDGE_VERTEX) | (1 << hhg.K_GHOST), L)
    for _ in range(reps):
        g.p2_apply(Lp, x, y, stream=st)
    torch.cuda.synchronize()
    _, kms = hhg.profile_end()
    ms = sum(kms) / reps
    N1 = info.N
    n_v = info.n_faces * (N1 // 2 - 1) * (N1 // 2 - 2) // 2       # micro-vertex face points
    n_all = info.n_faces * (N1 - 1) * (N1 - 2) // 2
    ops = 13.0 * n_v + 7.0 * (n_all - n_v)
    peak = n_sm * FP64_OPS_PER_CLK_SM * sm_mhz * 1e6 / 1e9
    ach = ops / (ms / 1e3) / 1e9
    return {"workload": f"annulus-128faces-P2-L{Lp} ({info.n_free} free P2 unknowns = the level-{L} lattice)",
            "solve": {"seconds": dt, "cycles": rep["iterations"], "rel_residual": rep["r_final"] / rep["r0"],
                      "factor_per_cycle": (rep["r_final"] / rep["r0"]) ** (1.0 / max(1, rep["iterations"])),
                      "gdofs_per_cycle": info.n_free * rep["iterations"] / dt / 1e9,
                      "cycle": "p-multigrid: P2 GS V(2,2) + one P1 V(3,3) on the same level"},
            "apply_roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "G FP64-instr/s",
                               "frac": ach / peak, "ms_per_apply": ms,
                               "hbm_gbs": 16.0 * info.n_free / (ms / 1e3) / 1e9, "hbm_peak_gbs": hbm_peak,
                               "model": "13 FP64 instr per micro-vertex point, 7 per edge point; 16 B per point"}}


def run_stokes(args, dev, st, hbm_peak, n_sm, sm_mhz):
    """Stokes flow, P1-P1 with PSPG stabilisation, by the all-at-once variable
    V(2,2) multigrid (two more steps per coarser level) with the inexact Uzawa
    smoother (delta 0.3, omega 0.4, two velocity sweeps per step, direct
    level-0 correction) on the 256-face annulus (32 sectors x 4 rings:
    micro-triangles of aspect ratio about 1.4; the 64 x 2 split's aspect ratio
    3 slows every pointwise smoother, the P1 Poisson cycle included): at the
    paper's energy-transport size (level 6, 2145 unknowns per macro-face) and
    at level 9.  Right-hand sides: SplitMix64 seeds 71, 72, 73 in canonical
    order, g shifted to zero sum.  Reported: time to a 1e-8 relative residual
    (the cycle replayed as a captured graph), cycles, factor, DoF rate over all
    three fields, and the roofline of the Stokes face-row kernels inside the
    smoother: FP64-instruction bound (11 + 24 instructions per face point and
    step), their HBM rate beside it."""
    import torch
    from paper_1805_10167_gb300 import hhg, inputs
    xy, tri = inputs.annulus_mesh(32, 4)
    out = {}
    for L in (6, 9):
        g = hhg.Mesh(xy, tri, L)
        g.stokes_setup(0.3, 0.4, 2, 0)
        info = g.info(L)
        vec = lambda: torch.zeros(info.vec_len, dtype=torch.float64, device=dev)  # noqa: E731
        rhs = []
        for seed in (71, 72, 73):
            c = torch.tensor(inputs.uniform_pm1(info.n_nodes, seed), dtype=torch.float64, device=dev)
            if seed == 73:
                c -= c.mean()
            v = vec()
            g.from_canonical(L, c, v, stream=st)
            rhs.append(v)
        u = [vec() for _ in range(3)]
        g.stokes_solve(L, *u, *rhs, tol=1e-8, max_iter=200, stream=st)     # warm-up: graph capture
        for v in u:
            v.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = g.stokes_solve(L, *u, *rhs, tol=1e-8, max_iter=200, stream=st)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dofs = 2 * info.n_free + info.n_nodes
        res = {"level": L, "macro_faces": info.n_faces, "dofs": dofs,
               "seconds_to_1e-8": dt, "cycles": rep["iterations"],
               "factor_per_cycle": (rep["r_final"] / rep["r0"]) ** (1.0 / max(1, rep["iterations"])),
               "ms_per_cycle": 1e3 * dt / max(1, rep["iterations"]),
               "gdofs_per_cycle": dofs * rep["iterations"] / dt / 1e9}
        # FP32 variable V-cycles inside FP64 iterative refinement, same tolerance
        for v in u:
            v.zero_()
        g.stokes_solve_ir(L, *u, *rhs, tol=1e-8, max_iter=200, stream=st)   # warm-up: buffers, graph capture
        for v in u:
            v.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep32 = g.stokes_solve_ir(L, *u, *rhs, tol=1e-8, max_iter=200, stream=st)
        torch.cuda.synchronize()
        dt32 = time.perf_counter() - t0
        res["fp32_ir"] = {"seconds_to_1e-8": dt32, "steps": rep32["iterations"],
                          "rel_residual": rep32["r_final"] / rep32["r0"],
                          "ms_per_step": 1e3 * dt32 / max(1, rep32["iterations"]),
                          "speedup_vs_fp64": dt / dt32}
        if L == 9:
            steps = 8
            g.stokes_smooth(L, *u, *rhs, forward=True, steps=2, stream=st)
            torch.cuda.synchronize()
            hhg.profile_begin(1 << hhg.K_FACE_ROWS, L)
            g.stokes_smooth(L, *u, *rhs, forward=True, steps=steps, stream=st)
            torch.cuda.synchronize()
            _, kms = hhg.profile_end()
            ms = sum(kms)
            pts = info.n_faces * (info.N - 1) * (info.N - 2) // 2
            ops = 35.0 * pts * steps
            peak = n_sm * FP64_OPS_PER_CLK_SM * sm_mhz * 1e6 / 1e9
            ach = ops / (ms / 1e3) / 1e9
            gbs = 88.0 * pts * steps / (ms / 1e3) / 1e9
            res["face_rows_roofline"] = {
                "bound": "alu", "achieved": ach, "peak": peak, "unit": "G FP64-instr/s", "frac": ach / peak,
                "ms_per_step": ms / steps, "hbm_gbs": gbs, "hbm_peak_gbs": hbm_peak,
                "model": "per Uzawa step and face point: gradient rows 11 FP64 instructions (read p, f1, f2, "
                         "write b1, b2: 40 B), pressure Jacobi rows 24 (read u1, u2, p, g, 1/s, write p: 48 B); "
                         "peak 2 FP64 instructions per clock per SM at the sampled clock"}
        out[f"L{L}"] = res
        g.close()
    out["workload"] = "annulus-32x4-256faces P1-P1 PSPG Stokes, all-at-once variable V(2,2) (+2 steps per coarser level), inexact Uzawa"
    return out


def vark_mesh(level, dev, st):
    """The 128-face annulus with k = exp(g), g the seeded (42) random field of
    squared-exponential covariance (length 0.1, sigma 1) at element centroids."""
    import torch

    from paper_1805_10167_gb300 import hhg, inputs
    xy, tri = inputs.annulus_mesh(32, 2)
    g = hhg.Mesh(xy, tri, level)
    k = inputs.grf_coefficient(inputs.element_centroids(xy, tri, level, device=dev), seed=42)
    g.set_coefficient(k, stream=st)
    del k
    info = g.info(level)
    bc = torch.tensor(inputs.uniform_pm1(info.n_nodes, 1234), dtype=torch.float64, device=dev)
    b = torch.zeros(info.vec_len, dtype=torch.float64, device=dev)
    g.from_canonical(level, bc, b, stream=st)
    return g, info, b


def timed_solve(g, level, b, st, **kw):
    import torch
    x = torch.zeros_like(b)
    g.solve(level, x, b, stream=st, **kw)          # warm-up
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, rep = g.solve(level, x, b, stream=st, **kw)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    it = rep["iterations"]
    return {"seconds": dt, "iterations": it, "rel_residual": rep["r_final"] / rep["r0"],
            "factor_per_iteration": (rep["r_final"] / rep["r0"]) ** (1.0 / max(it, 1)),
            "smoother_used": ["gs", "learned", "learned_gs"][rep.get("smoother_used", 0)],
            "judge": [rep.get("judge_learned", 0.0), rep.get("judge_gs", 0.0)]}


def run_vark(args, dev, st):
    """Variable-coefficient annulus, level 10: time to a 1e-10 relative FP64
    residual, FP64 V(3,3) against FP32 V(3,3) cycles inside FP64 iterative
    refinement."""
    from paper_1805_10167_gb300 import hhg
    L = args.level
    g, info, b = vark_mesh(L, dev, st)
    out = {"workload": f"annulus-128faces-L{L}-grf-k-V(3,3)", "free_dofs": info.n_free,
           "fp64_mg": timed_solve(g, L, b, st, mode=hhg.SOLVE_MG),
           "fp32_ir": timed_solve(g, L, b, st, mode=hhg.SOLVE_IR),
           "fp64_pcg": timed_solve(g, L, b, st, mode=hhg.SOLVE_PCG),
           "fp32_fpcg": timed_solve(g, L, b, st, mode=hhg.SOLVE_FPCG)}
    out["ir_speedup"] = out["fp64_mg"]["seconds"] / out["fp32_ir"]["seconds"]
    g.close()
    return out


def run_learned(args, dev, st):
    """Learned smoother on the variable-coefficient annulus at level 9: train
    on FP64 V-cycle residual/error crops, then FGMRES(20) preconditioned by
    one FP32 V(1,1) with the learned smoother alone, with a Gauss-Seidel sweep
    followed by the learned step (each judged, with fallback) or with
    Gauss-Seidel, against plain FP64 V(3,3) cycles."""
    from paper_1805_10167_gb300 import hhg
    L = max(6, args.level - 1)
    g, info, b = vark_mesh(L, dev, st)
    t0 = time.perf_counter()
    hist = g.learned_train(L, n_pairs=args.learned_pairs, epochs=args.learned_epochs, batch=128,
                           lr=1e-3, seed=0, stream=st)
    t_train = time.perf_counter() - t0
    out = {"workload": f"annulus-128faces-L{L}-grf-k", "free_dofs": info.n_free,
           "train_seconds": t_train, "train_pairs": args.learned_pairs, "epochs": args.learned_epochs,
           "loss_first_last": [float(hist[0]), float(hist[-1])] if len(hist) else None,
           "fgmres_learned": timed_solve(g, L, b, st, mode=hhg.SOLVE_FGMRES, nu1=1, nu2=1,
                                         smoother=hhg.SMOOTH_LEARNED),
           "fgmres_learned_gs": timed_solve(g, L, b, st, mode=hhg.SOLVE_FGMRES, nu1=1, nu2=1,
                                            smoother=hhg.SMOOTH_LEARNED_GS),
           "fgmres_gs": timed_solve(g, L, b, st, mode=hhg.SOLVE_FGMRES, nu1=1, nu2=1,
                                    smoother=hhg.SMOOTH_GS),
           "fp64_mg": timed_solve(g, L, b, st, mode=hhg.SOLVE_MG),
           "cnn_roofline": cnn_roofline(g, L, info, dev)}
    g.close()
    return out


def cnn_roofline(g, L, info, dev, reps=20):
    """The trained network applied on level L (face scale, clear and the
    tensor-core kernel), timed by CUDA events on the launching stream,
    against the measured dense BF16 peak; flops = the network's own
    2 (27 + 144) 16 + 2 * 144 multiply-adds per face-interior point (no halo
    recomputation or padding counted)."""
    import torch
    from paper_1805_10167_gb300 import hhg
    gen = torch.Generator(device=dev).manual_seed(99)
    s = torch.randn(info.vec_len, dtype=torch.float32, device=dev, generator=gen)
    d = torch.zeros_like(s)
    for _ in range(3):
        g.learned_apply(L, s, d=d, prec=hhg.F32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.learned_apply(L, s, d=d, prec=hhg.F32)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    pts = info.n_faces * (info.N - 1) * (info.N - 2) // 2
    tflops = 2 * (3 * 9 * 16 + 16 * 9 * 16 + 16 * 9) * pts / (ms / 1e3) / 1e12
    peak = _peaks().get("bf16_tflops")
    basis = "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst), of measured"
    if not peak:
        peak, basis = 1900.0, "1.9 PFLOP/s bf16 burst, of fallback"
    return {"bound": "tensor", "kernel": "k_cnn_smooth (3 layers, mma.sync BF16, FP32 accumulate)",
            "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
            "ms_per_application": ms, "peak_basis": basis}


def _peaks():
    """The measured peak rates of the GB300 (MEASURED_PEAKS.json), {} when absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each step is one oracle V(3,3) + residual norm on the level --cpu-level
    # sample of the same annulus (about 0.6 s at level 8), K steps after W
    steps, warm = max(1, args.steps), max(0, args.warmup)
    rate, nproc, spc = oracle_pool_rate(args.cpu_level, steps, warmup=warm)
    from oracle import mesh as om
    from paper_1805_10167_gb300 import inputs as _inp
    _xy, _tri = _inp.annulus_mesh(32, 2)
    _lv = om.Level(om.MacroMesh(_xy, _tri), args.cpu_level)
    n_free = int(_lv.free.sum())
    sample = (f"annulus 32x2 (128 faces) at level {args.cpu_level} ({n_free} free DoFs), FP64 V(3,3) + "
              f"residual norm, {steps} cycles after {max(1, warm)} warm-up on each of {nproc} host cores (one "
              f"single-threaded numpy/scipy oracle process per core, independent replicas)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": spc * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(args.level)[2], "level": args.level},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": nproc, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1805_10167_gb300 import hhg, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    L = args.level
    xy, tri, wname = workload(L)
    g = hhg.Mesh(xy, tri, L)
    info = g.info(L)
    n_free = info.n_free
    st = torch.cuda.current_stream()
    b_canon = torch.tensor(inputs.uniform_pm1(info.n_nodes, 1234), dtype=torch.float64, device=dev)
    b = torch.zeros(info.vec_len, dtype=torch.float64, device=dev)
    x = torch.zeros_like(b)
    r = torch.zeros_like(b)
    nrm = torch.zeros(1, dtype=torch.float64, device=dev)
    g.from_canonical(L, b_canon, b, stream=st)

    def step():
        g.vcycle(L, x, b, nu1=3, nu2=3, stream=st)
        g.residual(L, x, b, r, nrm, stream=st)

    def barrier():
        rank_barrier(world)

    def max_over_ranks(v):
        return rank_max(v, world, dev)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # timed region: K steps as a user runs them (the V-cycle replays the CUDA
    # graph the library captured during the warm-up)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    value = job_rate(world, n_free, args.steps, ms)
    # the same K steps again with the library's launch profiling on: every
    # launch is issued and counted one by one, and the level-L sweeps are
    # bracketed by CUDA events on the stream they run on
    hhg.profile_begin(1 << hhg.K_FACE_GS, L)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(st)
    for _ in range(args.steps):
        step()
    e3.record(st)
    torch.cuda.synchronize()
    launches, kms = hhg.profile_end()
    clk = clocks.stop()
    barrier()
    ms_profiled = max_over_ranks(e2.elapsed_time(e3))

    # dominant kernel: the three-colour face Gauss-Seidel sweep on level L
    # (6 launches per V(3,3) cycle).  For k = 1 each interior point costs 6
    # FP64 instructions (3 add, 3 fma) when the strip kernel reads the scaled
    # right-hand side b / A_pp (made once per cycle on this level), else 7
    # (one more mul), and 24 algorithmic bytes (read x and b, write x); the
    # sweep is FP64-pipe bound on GB300.
    gs_launches_L = (3 + 3) * args.steps
    gs_ms = kms[hhg.K_FACE_GS] / gs_launches_L
    pts = info.n_faces * (info.N - 1) * (info.N - 2) // 2
    variant, split = g.sweep_config(L, hhg.F64)
    ops_per_point = 6.0 if variant == hhg.SWEEP_STRIP and info.N > 64 else 7.0
    ops = ops_per_point * pts
    sm_mhz = clk.get("sm_mhz") or 2070.0
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = n_sm * FP64_OPS_PER_CLK_SM * sm_mhz * 1e6 / 1e9        # G FP64 instr/s at the sampled clock
    achieved = ops / (gs_ms / 1e3) / 1e9
    bytes_alg = 24.0 * pts
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    kname = ("k_gs_sweep<double> whole sweep (vertices, edge colours, register-strip faces, %d-row tasks)" % split
             if variant == hhg.SWEEP_STRIP
             else "k_face_gs3<double> shared-memory ring sweep, %d row blocks per face" % split)
    # DRAM traffic of one launch from the ncu capture of this kernel at level 9
    # (profiles/), scaled by the points of level L
    traffic = TRAFFIC_L9.get((variant, split))
    if traffic is not None:
        traffic *= pts / 16760832.0
    roofline = {"bound": "alu", "kernel": f"{kname}, level {L}",
                "achieved": achieved, "peak": peak, "unit": "G FP64-instr/s", "frac": achieved / peak,
                "traffic": traffic, "ops_per_launch": ops, "ops_per_point": ops_per_point, "ms_per_launch": gs_ms,
                "peak_basis": f"{n_sm} SMs x {FP64_OPS_PER_CLK_SM} FP64 instr/clk x {sm_mhz:.0f} MHz (sampled)",
                "hbm": {"achieved_gbs": bytes_alg / (gs_ms / 1e3) / 1e9, "peak_gbs": hbm_peak,
                        "frac": bytes_alg / (gs_ms / 1e3) / 1e9 / hbm_peak,
                        "algorithmic_bytes_per_launch": bytes_alg}}

    # where a step's time goes: the same steps once more with every launch of
    # every class and level bracketed by CUDA events (the events add a little)
    hhg.profile_begin((1 << hhg.K_COUNT) - 1, -1)
    e2.record(st)
    for _ in range(args.steps):
        step()
    e3.record(st)
    torch.cuda.synchronize()
    _, cls_ms = hhg.profile_end()
    breakdown = {"ms_per_step_by_class": {nm: v / args.steps for nm, v in zip(hhg.K_NAMES, cls_ms)},
                 "ms_per_step": e2.elapsed_time(e3) / args.steps,
                 "note": "every launch of every level event-bracketed; the rest of ms_per_step is "
                         "launch gaps and copies"}

    # the FP32 V(3,3) (the inner cycle of refinement and flexible CG) on the
    # same level, and its face sweep: HBM-bound, against half the FP64 byte
    # model (144 B per free DoF per V(3,3) cycle, 12 B per sweep point)
    b32 = b.float()
    x32 = torch.zeros_like(b32)
    for _ in range(args.warmup):
        g.vcycle(L, x32, b32, nu1=3, nu2=3, prec=hhg.F32, stream=st)
    torch.cuda.synchronize()
    e2.record(st)
    for _ in range(args.steps):
        g.vcycle(L, x32, b32, nu1=3, nu2=3, prec=hhg.F32, stream=st)
    e3.record(st)
    torch.cuda.synchronize()
    ms32 = e2.elapsed_time(e3) / args.steps
    hhg.profile_begin(1 << hhg.K_FACE_GS, L)
    for _ in range(args.steps):
        g.vcycle(L, x32, b32, nu1=3, nu2=3, prec=hhg.F32, stream=st)
    torch.cuda.synchronize()
    _, kms32 = hhg.profile_end()
    sweep32_ms = kms32[hhg.K_FACE_GS] / (6 * args.steps)
    hbm_cycle = 144.0 * n_free / (ms32 / 1e3) / 1e9
    hbm_sweep = 12.0 * pts / (sweep32_ms / 1e3) / 1e9
    fp32_vcycle = {"gdofs": n_free / (ms32 / 1e3) / 1e9, "ms_per_cycle": ms32,
                   "roofline": {"bound": "hbm", "achieved": hbm_cycle, "peak": hbm_peak, "unit": "GB/s",
                                "frac": hbm_cycle / hbm_peak,
                                "model": "144 B per free DoF per V(3,3) cycle (half the FP64 cycle's 288)"},
                   "sweep": {"ms_per_launch": sweep32_ms, "achieved_gbs": hbm_sweep, "frac": hbm_sweep / hbm_peak,
                             "model": "12 B per face-interior point (read x, b; write x)"}}
    del b32, x32

    # end to end through the public API from pinned host memory: every step
    # uploads b and reads back the iterate x (canonical order) and the norm
    b_host = b_canon.cpu().pin_memory()
    nrm_host = torch.zeros(1, dtype=torch.float64).pin_memory()
    x_hosts = [torch.empty(info.n_nodes, dtype=torch.float64).pin_memory() for _ in range(2)]
    x.zero_()
    # Two staging vectors per direction, two device right-hand sides and two
    # copy streams: the host->device copy of step k + 1's right-hand side and
    # its conversion to the internal layout (into the right-hand side step k
    # does not read), and the device->host copy of step k - 1's iterate, run
    # while step k computes.  A buffer is reused only after the step or copy
    # that last read it.
    up_st = torch.cuda.Stream(device=dev)
    down_st = torch.cuda.Stream(device=dev)
    stages = [torch.empty_like(b_canon), torch.empty_like(b_canon)]
    xstages = [torch.empty_like(b_canon), torch.empty_like(b_canon)]
    bdev = [b, torch.zeros_like(b)]
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    freed = [torch.cuda.Event(), torch.cuda.Event()]
    produced = [torch.cuda.Event(), torch.cuda.Event()]
    downloaded = [torch.cuda.Event(), torch.cuda.Event()]

    def upload(k):
        s = k % 2
        up_st.wait_event(freed[s])
        with torch.cuda.stream(up_st):
            stages[s].copy_(b_host, non_blocking=True)
        g.from_canonical(L, stages[s], bdev[s], stream=up_st)
        ready[s].record(up_st)

    def e2e_steps(n):
        for ev in freed + downloaded:
            ev.record(st)
        upload(0)
        for k in range(n):
            if k + 1 < n:
                upload(k + 1)
            s = k % 2
            st.wait_event(ready[s])
            g.vcycle(L, x, bdev[s], nu1=3, nu2=3, stream=st)
            g.residual(L, x, bdev[s], r, nrm, stream=st)
            freed[s].record(st)
            nrm_host.copy_(nrm, non_blocking=True)
            st.wait_event(downloaded[s])
            g.to_canonical(L, x, xstages[s], stream=st)
            produced[s].record(st)
            down_st.wait_event(produced[s])
            with torch.cuda.stream(down_st):
                x_hosts[s].copy_(xstages[s], non_blocking=True)
            downloaded[s].record(down_st)
        st.wait_stream(down_st)
        st.wait_stream(up_st)

    e2e_steps(max(args.warmup, 6))    # each device right-hand side's cycle graph is captured on its third use
    torch.cuda.synchronize()
    barrier()
    e0.record(st)
    e2e_steps(args.steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1))
    assert bool(torch.isfinite(x_hosts[(args.steps - 1) % 2]).all())
    e2e = {"value": job_rate(world, n_free, args.steps, ms_e2e), "unit": UNIT,
           "h2d_bytes_per_step": int(b_host.numel() * 8),
           "d2h_bytes_per_step": int(info.n_nodes * 8 + 8),
           "ms_per_step": ms_e2e / args.steps,
           "pipeline": "each step: pinned host b -> device and canonical -> internal layout (copy "
                       "stream, into the second device right-hand side, overlapping the previous step), "
                       "V(3,3), residual norm -> pinned host, iterate x -> canonical order -> pinned host "
                       "(second copy stream, overlapping the next step)"}
    del x_hosts, xstages, stages, bdev

    # time to a 1e-10 relative FP64 residual: FP64 MG vs FP32-in-FP64 IR
    solve = None
    if not args.no_solve:
        solve = {}
        for name, mode in (("fp64_mg", hhg.SOLVE_MG), ("fp32_ir", hhg.SOLVE_IR), ("fp64_pcg", hhg.SOLVE_PCG),
                           ("fp32_fpcg", hhg.SOLVE_FPCG)):
            x.zero_()
            g.solve(L, x, b, mode=mode, stream=st)          # warm-up
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, rep = g.solve(L, x, b, mode=mode, stream=st)
            torch.cuda.synchronize()
            solve[name] = {"seconds": time.perf_counter() - t0, "cycles": rep["iterations"],
                           "rel_residual": rep["r_final"] / rep["r0"]}

    p2res = None if args.no_p2 else run_p2(args, g, info, b, dev, st, hbm_peak, n_sm, sm_mhz)
    g.close()
    batch = None if args.no_batch else run_batch(args, dev, st)
    vark = None if args.no_vark else run_vark(args, dev, st)
    learned_res = None if args.no_learned else run_learned(args, dev, st)
    stokes_res = None if args.no_stokes else run_stokes(args, dev, st, hbm_peak, n_sm, sm_mhz)

    fp64_probe = fp64_dgemm_probe(dev)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate1, spc, nf = oracle_rate(args.cpu_level, 8)
        rate_all, nproc, spc_all = oracle_pool_rate(args.cpu_level, 8)
        mg_cycles = solve["fp64_mg"]["cycles"] if solve else 13
        # one C2 problem in the oracle: single-threaded, cost proportional to
        # the unknowns (measured per cycle at the sample level), times the
        # cycles the same V(3,3) needs at C2 (the GPU's count: same method)
        t_tol = spc * (n_free / nf) * (mg_cycles + 1)
        cpu = {"value": rate_all, "unit": UNIT, "cores": nproc, "kind": "oracle",
               "sample": f"annulus 32x2 at level {args.cpu_level} ({nf} free DoFs), FP64 V(3,3) + residual norm, "
                         f"8 cycles on each of {nproc} host cores (one single-threaded numpy/scipy oracle "
                         f"process per core, independent replicas, spawn), {spc_all:.2f} s/cycle per process",
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1, "seconds_per_cycle": spc},
               "time_to_tol_extrapolated_s": {
                   "value": t_tol, "cycles": mg_cycles,
                   "basis": f"oracle single thread, {spc:.2f} s per cycle at level {args.cpu_level} scaled by "
                            f"{n_free}/{nf} unknowns, {mg_cycles} V(3,3) cycles + the initial residual "
                            f"(the count the same method needs at level {L}); extrapolated, not run"}}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "level": L, "macro_faces": info.n_faces, "free_dofs": n_free,
                       "cycle": "V(3,3), 3-colour GS, direct level-0 solve", "rhs": "SplitMix64 seed 1234",
                       "parallelism": f"replicas x{world}",
                       "launch": "V-cycle replayed as a captured CUDA graph; residual launched directly",
                       "l2": "inputs larger than L2 (%.2f GB per level-%d vector)" % (info.vec_len * 8 / 1e9, L)},
            "clocks": clk, "e2e": e2e, "gpu_launches": int(sum(launches)),
            "launches_by_class": dict(zip(hhg.K_NAMES, launches)),
            "profiled_pass": {"ms_per_step": ms_profiled / args.steps,
                              "note": "the same steps with every launch issued and counted one by one; "
                                      "gpu_launches and the roofline kernel time come from this pass"},
            "roofline": roofline, "breakdown": breakdown, "fp32_vcycle": fp32_vcycle,
            "fp64_peak_probe": fp64_probe, "cpu_baseline": cpu, "time_to_tol": solve, "batch": batch,
            "vark": vark, "learned": learned_res, "p2": p2res, "stokes": stokes_res,
        }), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_sweep_case(args):
    """Four forward Gauss-Seidel sweeps of level --level of the 128-face
    annulus in --prec with the default kernel configuration (inputs, output
    and workspace above the 129 MB L2 from level 9 on); in FP64 they read
    b / A_pp made by one scaling pass first, as inside a V-cycle."""
    import torch
    from paper_1805_10167_gb300 import hhg, inputs
    xy, tri = inputs.annulus_mesh(32, 2)
    g = hhg.Mesh(xy, tri, args.level)
    g.fp64_arith(hhg.ARITH_DFLOAT if args.arith == "dfloat" else hhg.ARITH_IEEE)
    prec = hhg.F64 if args.prec == "f64" else hhg.F32
    info = g.info(args.level)
    dt = torch.float64 if prec == hhg.F64 else torch.float32
    gen = torch.Generator(device="cuda").manual_seed(1234)
    x = torch.rand(info.vec_len, dtype=dt, device="cuda", generator=gen)
    b = torch.rand(info.vec_len, dtype=dt, device="cuda", generator=gen)
    g.smooth(args.level, x, b, hhg.GS_FWD, sweeps=4, prec=prec)
    torch.cuda.synchronize()
    g.close()
    print("sweep case done")


def run_cnn_case(args):
    """The learned smoother's network on every face of level --level of the
    variable-coefficient 128-face annulus, on each tensor-core path
    (k_cnn_smooth, then k_cnn_smooth_tc): --warmup untimed and --steps timed
    applications to a random FP32 scaled residual, with seeded random weights
    (the cost does not depend on their values)."""
    import torch
    from paper_1805_10167_gb300 import hhg
    dev = torch.device("cuda:0")
    L = args.level
    g, info, _ = vark_mesh(L, dev, None)
    rng = np.random.default_rng(0)
    g.learned_set_weights((0.1 * rng.standard_normal(hhg.LEARNED_NPARAMS)).astype(np.float32))
    gen = torch.Generator(device="cuda").manual_seed(1234)
    s = torch.randn(info.vec_len, dtype=torch.float32, device=dev, generator=gen)
    d = torch.zeros_like(s)
    pts = info.n_faces * (info.N - 1) * (info.N - 2) // 2
    flop = 2 * (3 * 9 * 16 + 16 * 9 * 16 + 16 * 9 * 1) * pts
    for name, path in (("mma.sync", hhg.TC_MMA_SYNC), ("tcgen05 layer 2", hhg.TC_TCGEN05)):
        g.learned_tensor_path(path)
        for _ in range(args.warmup):
            g.learned_apply(L, s, d=d, prec=hhg.F32)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            g.learned_apply(L, s, d=d, prec=hhg.F32)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(args.steps, 1)
        print(f"cnn case ({name}): level {L}, {pts} face-interior points, {ms:.3f} ms per application "
              f"(face scale, clear, network), {flop / ms / 1e9:.1f} TFLOP/s of the network's own flops")
    g.learned_tensor_path(hhg.TC_MMA_SYNC)
    g.close()


def run_stokes_case(args):
    """--warmup untimed and --steps timed forward Uzawa steps of the Stokes
    smoother on level --level of the 256-face annulus (every level vector above
    the 129 MB L2 from level 9 on), with the per-class event timing of the
    Stokes face-row kernels printed; no JSON line."""
    import torch
    from paper_1805_10167_gb300 import hhg, inputs
    xy, tri = inputs.annulus_mesh(32, 4)
    L = args.level
    g = hhg.Mesh(xy, tri, L)
    g.stokes_setup()
    info = g.info(L)
    gen = torch.Generator(device="cuda").manual_seed(1234)
    v = [torch.rand(info.vec_len, dtype=torch.float64, device="cuda", generator=gen) for _ in range(6)]
    g.stokes_smooth(L, *v, forward=True, steps=args.warmup)
    torch.cuda.synchronize()
    hhg.profile_begin(1 << hhg.K_FACE_ROWS, L)
    g.stokes_smooth(L, *v, forward=True, steps=args.steps)
    torch.cuda.synchronize()
    _, kms = hhg.profile_end()
    pts = info.n_faces * (info.N - 1) * (info.N - 2) // 2
    ms = sum(kms)
    print(f"stokes case done: face rows {ms / args.steps:.3f} ms per step, "
          f"{35.0 * pts * args.steps / (ms / 1e3) / 1e9:.0f} G FP64-instr/s, "
          f"{88.0 * pts * args.steps / (ms / 1e3) / 1e9:.0f} GB/s algorithmic")
    g.close()


if __name__ == "__main__":
    a = parse()
    if a.case == "stokes":
        run_stokes_case(a)
    elif a.case == "sweep":
        run_sweep_case(a)
    elif a.case == "cnn":
        run_cnn_case(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
