"""SSAMG-PCG benchmark on one GB300 (or N replicas, one per GPU).

Workload (default): 8 parts of 64^3 cells in a 2x2x2 layout (2,097,152
unknowns), 7-point anisotropic diffusion with per-part (a_x, a_y, a_z) ~
log-uniform[1e-3, 1] (seed 1), harmonic-mean inter-part couplings, RHS ~
U[-1,1]; PCG with one SSAMG V(1,1) cycle per iteration from x0 = 0 to a
1e-8 relative residual.  A step is one SSAMG setup plus one PCG solve, with
the assembled matrix already resident on the device.  The headline uses the
FP32 V-cycle inside FP64 PCG; the plain FP64 method is timed the same way and
reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs its own replica of the workload (no data-path
collective; barrier and max-over-ranks timing only).  --impl reference times
the CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import problems as P  # noqa: E402

METRIC = "SSAMG-PCG setup+solve ms, MDOF/s to 1e-8 rel. res., FP32-cycle vs FP64; %HBM"
WORKLOAD = "8 parts x 64^3 (2x2x2 layout), 7-pt anisotropic diffusion, seed 1"
L2_BYTES = 129 * 2 ** 20


def max_over_ranks(value, ws, device=None):
    """The largest of the ranks' values (a replicated job takes as long as its
    slowest rank); every rank gets it.  One rank: the value itself."""
    if ws == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mdof_s(n_per_rank, ws, step_ms):
    """Whole-job throughput of ws replicas of an n_per_rank-unknown step
    (weak scaling): all ranks' unknowns over the slowest rank's time."""
    return ws * n_per_rank / (step_ms * 1e-3) / 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        load = [s for s in sm if mx and s > 0.3 * max(mx)] or sm
        out["sm_mhz"] = statistics.median(load) if load else None
        out["sm_max_mhz"] = max(mx) if mx else None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


def fmt(v):
    if isinstance(v, float):
        return float(f"{v:.4e}") if 0 < abs(v) < 1e-3 else round(v, 4)
    return v


def flush_l2(buf):
    buf.add_(1.0)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2205_14273_gb300 import ssamg as S

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    S.lib()

    prob = P.config(1)
    N = prob.n
    grid, A = S.matrix_from_problem(prob)
    b = torch.as_tensor(prob.b[0], device=dev)
    x = torch.zeros_like(b)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def make(precision):
        return S.Solver(precision=precision, flexible=precision, tol=1e-8, max_iter=500,
                        use_graph=0 if args.no_graph else 1)

    solvers = {"fp32_cycle": make(1), "fp64": make(0)}
    if args.only:
        solvers = {args.only: solvers[args.only]}
    results = {}
    for name, sv in solvers.items():
        # warm-up steps (also builds the arena and the CUDA graph)
        for _ in range(args.warmup):
            sv.setup(A)
            sv.solve(b, x)
        table = None
        if args.autotune:
            table = sv.autotune(reps=20)
            sv.setup(A)
            sv.solve(b, x)
        st = sv.solve(b, x)
        assert st.converged and st.true_rel_res <= 1.05e-8, (name, st.as_dict())
        verified = st.as_dict()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        clocks = ClockSampler(local)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush_l2(flush)
            e0, e1, e2 = ev[k]
            e0.record(stream)
            sv.setup(A)
            e1.record(stream)
            sv.solve_nostats(b, x)
            e2.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if ws > 1:
            dist.barrier()
        ck = clocks.stop()
        setup_ms = [e0.elapsed_time(e1) for e0, e1, _ in ev]
        solve_ms = [e1.elapsed_time(e2) for _, e1, e2 in ev]
        step_ms = max_over_ranks(sum(setup_ms) / args.steps + sum(solve_ms) / args.steps, ws, dev)
        results[name] = {
            "ms_per_step": step_ms,
            "setup_ms": statistics.median(setup_ms),
            "solve_ms": statistics.median(solve_ms),
            "iterations": verified["iterations"],
            "true_rel_res": verified["true_rel_res"],
            "levels": verified["num_levels"],
            "operator_complexity": verified["operator_complexity"],
            "launches": int(verified["setup_kernel_launches"] + verified["solve_kernel_launches"]),
            "mdof_s": job_mdof_s(N, ws, step_ms),
            "solve_mdof_s": job_mdof_s(N, ws, statistics.median(solve_ms)),
            "wall_s": wall,
            "clocks": ck,
        }
        if table is not None:
            results[name]["tile_table"] = tile_summary(table)

    if args.levels:
        for name, sv in solvers.items():
            level_table(sv, name, stream)

    # ---- dominant-kernel roofline (restriction with the fused pre-relaxation, FP32 cycle)
    roof = kernel_roofline(S, next(iter(solvers.values())), prob, dev, stream, args)

    # ---- per-kernel HBM fractions on the large levels, and the other two
    # full-size workloads
    peak = read_peaks().get("hbm_gbs", 6800.0)
    hbm = hbm_by_level(solvers.get("fp32_cycle", next(iter(solvers.values()))),
                       "8 parts x 64^3", stream, peak)
    extra = None if args.no_extra_workloads else extra_workloads(S, stream, peak)

    # ---- end to end through the C ABI with host buffers (matrix upload,
    # setup, solve, result read-back)
    e2e = None if args.no_e2e else end_to_end(S, prob, dev, stream, args)

    head = results.get("fp32_cycle") or results["fp64"]
    other = results.get("fp64", head)
    line = {
        "metric": METRIC,
        "value": round(head["mdof_s"], 3),
        "unit": "MDOF/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(head["ms_per_step"], 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32-cycle/f64-pcg",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "unknowns": N, "tol": 1e-8, "parallelism": f"replicas{ws}",
                   "l2": "flushed between steps (write of 2x L2)"},
        "setup_ms": round(head["setup_ms"], 4),
        "solve_ms": round(head["solve_ms"], 4),
        "iterations": head["iterations"],
        "fp64": {k: fmt(v) for k, v in other.items() if k != "clocks"},
        "fp32_cycle": {k: fmt(v) for k, v in head.items() if k != "clocks"},
        "speedup_fp32_cycle_vs_fp64": round(other["ms_per_step"] / head["ms_per_step"], 3),
        "gpu_launches": None,
        "roofline": roof,
        "e2e": e2e,
        "clocks": head["clocks"],
        "hbm_by_level": hbm,
    }
    if extra is not None:
        line["other_workloads"] = extra
    line["gpu_launches"] = head["launches"]
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def kernel_roofline(S, sv, prob, dev, stream, args):
    """Roofline of the dominant kernel of the timed step.

    The restriction (k_restrict, which on every level above the coarsest
    also does the coarse level's pre-relaxation with its U x row jobs) has
    the largest share of the step in the launch list, the prolongation with
    U x (k_prolong_u) the next; both run once per level and cycle.
    achieved = the kernel's algorithmic bytes summed over the levels of one
    V-cycle / its summed launch durations, each measured with CUDA events
    around graph replays of that launch on this stream.  Bytes per level
    (FP32 cycle, w = 4): restriction: fine residual (w N_l), P weights
    (2 w per fine point), coarse right-hand side out (w N_{l+1}) and, when
    fused, omega M^-1 in and x out (2 w N_{l+1}) and the coarse level's
    coupling rows (12 per row) and couplings (44 each: column, value,
    restriction row of the column, its diagonal, three fine residuals);
    prolongation: x in + x out (8 N_l), coarse correction (4 N_{l+1}),
    P weights (8 per fine point), coupling rows (12 per row) and couplings
    (36 each: column, value, P row of the column, x and two coarse values).
    """
    peaks = read_peaks()
    L = sv.num_levels()
    sizes = [sv.level_sizes(l) for l in range(L)]
    w = 4

    def restrict_bytes(l):
        N = sizes[l][0]
        Nc, nrc, nnzc = sizes[l + 1]
        pre = 2 * w * Nc + 12 * nrc + 44 * nnzc if l + 2 < L else 0
        return w * N + w * Nc + 2 * w * (N - Nc) + pre

    def prolong_bytes(l):
        N, nr, nnz = sizes[l]
        Nc = sizes[l + 1][0]
        return 8 * N + 4 * Nc + 8 * (N - Nc) + 12 * nr + 36 * nnz

    peak = peaks.get("hbm_gbs", 6800.0)

    def over_levels(kid, nbytes, name):
        tot_us = tot_b = 0.0
        per_level = []
        for l in range(L - 1):
            us = sv.time_kernel(kid, l, 50, stream)
            tot_us += us
            tot_b += nbytes(l)
            per_level.append(round(us, 2))
        nl = L - 1
        achieved = tot_b / (tot_us * 1e-6) / 1e9
        return {
            "kernel": name,
            "bound": "hbm",
            "achieved": round(achieved, 1),
            "peak": peak,
            "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
            "traffic": None,
            "bytes_per_launch": int(tot_b / nl),
            "us_per_launch": round(tot_us / nl, 3),
            "us_per_level": per_level,
        }

    out = over_levels(3, restrict_bytes,
                      "k_restrict<float> (restriction P^T r, with the coarse level's "
                      "pre-relaxation and U x row jobs), all levels of one V-cycle")
    out["second_kernel"] = over_levels(
        4, prolong_bytes,
        "k_prolong_u<float> (prolongation x + P e with U x row jobs), all levels of one V-cycle")
    # the FP64 level-0 operator apply + dot (the PCG's largest single launch)
    us_spmv = sv.time_kernel(6, 0, 50, stream)
    N0 = sizes[0][0]
    flops = 2 * 8 * N0 + 2 * prob.nnz_u
    out["fp64_level0_operator"] = {
        "kernel": "k7b_spmv_dot (q = A p and p.q, FP64, level 0 bricks)",
        "bound": "alu", "unit": "TFLOP/s",
        "achieved": round(flops / (us_spmv * 1e-6) / 1e12, 4),
        "peak": 1.25, "peak_source": "nominal GB300 FP64; 1.255 measured by an FMA probe",
        "frac": round(flops / (us_spmv * 1e-6) / 1.25e12, 4),
        "us_per_launch": round(us_spmv, 2),
        "hbm_gbs": round((24 * N0 + 16 * prob.nnz_u) / (us_spmv * 1e-6) / 1e9, 1)}
    return out


def level_table(sv, name, stream):
    """Per-level duration (us) of each cycle kernel, each timed alone as 100
    graph-replayed launches on the solver's own buffers (stderr).  The
    restriction onto a level above the coarsest also does that level's
    pre-relaxation (the "restrict" column of level l times the launch that
    restricts onto l + 1), so the cycle runs the separate pre-relaxation on
    level 0 only."""
    kinds = [("relax0_u", 2), ("residual", 0), ("restrict", 3), ("prolong_u", 4),
             ("relax", 1)]
    L = sv.num_levels()
    out = [f"{name}: PCG iteration {sv.time_kernel(7, 0, 20, stream):.1f} us = V-cycle "
           f"{sv.time_kernel(5, 0, 20, stream):.1f} us + FP64 operator apply "
           f"{sv.time_kernel(6, 0, 50, stream):.1f} us + vector steps "
           f"{sv.time_kernel(8, 0, 50, stream):.1f} us (+ U x of p)"
           + (f"; last relaxation as the PCG runs it {sv.time_kernel(9, 0, 50, stream):.1f} us"
              if name.startswith("fp32") else "")]
    out.append("  lvl        N     nr " + " ".join(f"{k:>11s}" for k, _ in kinds))
    for l in range(L):
        n, nr, _ = sv.level_sizes(l)
        row = []
        for _, kid in kinds:
            if (kid in (3, 4) and l == L - 1) or (kid == 2 and l > 0):
                row.append("-")
            else:
                row.append(f"{sv.time_kernel(kid, l, 100, stream):.2f}")
        out.append(f"  {l:3d} {n:8d} {nr:6d} " + " ".join(f"{v:>11s}" for v in row))
    print("\n".join(out), file=sys.stderr)


def hbm_by_level(sv, workload, stream, peak, min_cells=1 << 20):
    """Per-kernel HBM throughput of the FP32 cycle on the levels of at least
    2^20 cells: algorithmic bytes (each input and output once; w = 4) / the
    kernel's CUDA-graph launch time (50 replayed launches on the solver's own
    buffers), against the measured copy bandwidth.  Launches moving less than
    ~3/4 of L2 are flagged l2_resident."""
    w = 4
    L = sv.num_levels()
    sizes = [sv.level_sizes(l) for l in range(L)]
    rows = []
    for l in range(L - 1):
        N, nr, nnz = sizes[l]
        if N < min_cells:
            continue
        Nc, nrc, nnzc = sizes[l + 1]
        sc = sv.stored_coefficients(l)
        # the restriction onto a level above the coarsest also pre-relaxes it:
        # omega M^-1 read, x written, and its U x rows (structure, the
        # columns' restriction rows and diagonals, three fine residuals each)
        pre = 2 * w * Nc + 12 * nrc + 44 * nnzc if l + 2 < L else 0
        nbytes = {
            "relax0_u": (2, 3 * w * N + 12 * nr + 12 * nnz),
            "residual": (0, w * (sc + 3 * N)),
            "restrict": (3, w * N + w * Nc + 2 * w * (N - Nc) + pre),
            "prolong_u": (4, 2 * w * N + w * Nc + 2 * w * (N - Nc) + 12 * nr + 36 * nnz),
            "relax": (1, w * (sc + 4 * N)),
        }
        row = {"level": l, "cells": N, "stored_coefficients": sc}
        if l > 0:
            del nbytes["relax0_u"]  # done by the restriction onto this level
        for k, (kid, nb) in nbytes.items():
            us = sv.time_kernel(kid, l, 50, stream)
            gbs = nb / (us * 1e-6) / 1e9
            row[k] = {"us": round(us, 2), "gbs": round(gbs, 1), "frac": round(gbs / peak, 3)}
            if nb < 0.75 * L2_BYTES:
                # replayed launches of a kernel this small find their data in
                # the 129 MB L2: the fraction is of the HBM copy rate, the
                # bytes are mostly served by L2
                row[k]["l2_resident"] = True
        rows.append(row)
    return {"workload": workload, "peak_gbs": peak, "levels": rows}


def tile_summary(table):
    """Non-default entries of a tile table: size class -> form."""
    return {f"2^{c}": (f"{t & 7} cells/thread" + (" + bricks" if t & 8 else ""))
            for c, t in enumerate(table) if t}


def extra_workloads(S, stream, peak):
    """The 256^3 27-point workload and the 64-problem batched workload at full
    size: setup and solve times (one step after a warm-up) in both cycle
    precisions, and the per-kernel HBM fractions of their large levels; and
    the 128^3 differentiation workload."""
    import torch
    out = {}
    prob = P.config(2)
    grid, A = S.matrix_from_problem(prob)
    b = torch.as_tensor(prob.b[0], device="cuda")
    res = {"workload": "1 part 256^3, 27-point variable coefficients, seed 2",
           "unknowns": prob.n}
    for prec, name in ((1, "fp32_cycle"), (0, "fp64")):
        sv = S.Solver(precision=prec, flexible=prec, tol=1e-8, max_iter=500)
        sv.setup(A)
        x = torch.zeros_like(b)
        st = sv.solve(b, x)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        sv.setup(A)
        e[1].record(stream)
        sv.solve_nostats(b, x)
        e[2].record(stream)
        torch.cuda.synchronize()
        t_s, t_v = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
        res[name] = {"setup_ms": round(t_s, 3), "solve_ms": round(t_v, 3),
                     "iterations": st.iterations, "true_rel_res": fmt(st.true_rel_res),
                     "levels": st.num_levels,
                     "mdof_s": round(prob.n / ((t_s + t_v) * 1e-3) / 1e6, 3)}
        if prec == 1:
            res["hbm"] = hbm_by_level(sv, res["workload"], stream, peak)
    out["var27_256"] = res
    del A, grid
    probs = P.config(3)
    mats = [S.matrix_from_problem(p) for p in probs]
    nrhs = probs[0].b.shape[0]
    res = {"workload": f"{len(probs)} problems, 1-8 chained parts each, edges 16-96, "
                       f"{nrhs} right-hand sides, seed 3"}
    for prec, name in ((1, "fp32_cycle"), (0, "fp64")):
        B = S.Batch([A for _, A in mats], precision=prec, flexible=prec, tol=1e-8, max_iter=500)
        off = B.offsets()
        bh = np.zeros((nrhs, off[-1]))
        for k, p in enumerate(probs):
            bh[:, off[k]:off[k + 1]] = p.b
        bb = torch.as_tensor(bh, device="cuda")
        xx = torch.zeros_like(bb)
        B.setup()
        st = B.solve(bb, xx, nrhs)

        def timed():
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            B.setup()
            e[1].record(stream)
            st = B.solve(bb, xx, nrhs)
            e[2].record(stream)
            torch.cuda.synchronize()
            return st, e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])

        # built-in tiles, then the autotuner's table (the reported step)
        _, u_s, u_v = timed()
        t0 = time.perf_counter()
        table = B.autotune(reps=10)
        tune_s = time.perf_counter() - t0
        B.solve(bb, xx, nrhs)
        st, t_s, t_v = timed()
        its = [s.iterations for row in st for s in row]
        res["unknowns"] = off[-1]
        res[name] = {"setup_ms": round(t_s, 3), "solve_ms": round(t_v, 3),
                     "tile_table": tile_summary(table), "autotune_s": round(tune_s, 2),
                     "builtin_tiles": {"setup_ms": round(u_s, 3), "solve_ms": round(u_v, 3)},
                     "iterations_max": max(its), "iterations_mean": round(float(np.mean(its)), 2),
                     "worst_true_rel_res": fmt(max(s.true_rel_res for row in st for s in row)),
                     "levels": st[0][0].num_levels,
                     "mdof_s": round(off[-1] * nrhs / ((t_s + t_v) * 1e-3) / 1e6, 3)}
        if prec == 1:
            res["hbm"] = hbm_by_level(B.solver(), res["workload"], stream, peak)
        del B
    out["batched_64"] = res
    out["diffusion_128"] = differentiation_workload(S, stream, peak)
    return out


def differentiation_workload(S, stream, peak):
    """The differentiation form at full size (128^3, kappa = exp(g), FP64):
    setup, forward solve, adjoint solve A lambda = x - x_t on the same
    hierarchy, and dL/dg, each timed with CUDA events after a warm-up step;
    the gradient kernels' HBM fractions (k_diffusion_exp_gradient: g, lambda,
    x in and dL/dg out, 32 B per cell; k_coef_gradient: lambda and x in, the
    7 entries' dL/da out, 72 B per cell)."""
    import torch
    prob = P.config(4)
    N = prob.n
    grid, A = S.matrix_from_problem(prob)
    sv = S.Solver(tol=1e-8, max_iter=500)
    bt = torch.as_tensor(prob.b[0], device="cuda")
    xt = torch.as_tensor(prob.extra["x_t"], device="cuda")
    gt = torch.as_tensor(prob.extra["g"].reshape(-1), device="cuda")
    x = torch.zeros_like(bt)
    lam = torch.zeros_like(bt)
    dg = torch.zeros_like(bt)
    dcoef = torch.zeros(7 * N, dtype=torch.float64, device="cuda")

    def step(ev=None):
        mark = (lambda k: ev[k].record(stream)) if ev else (lambda k: None)
        mark(0)
        sv.setup(A)
        mark(1)
        st_f = sv.solve(bt, x)
        mark(2)
        st_a = sv.adjoint_solve(x - xt, lam)
        mark(3)
        sv.diffusion_exp_gradient(gt, lam, x, dg)
        mark(4)
        return st_f, st_a

    step()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    st_f, st_a = step(ev)
    torch.cuda.synchronize()
    t = [ev[k].elapsed_time(ev[k + 1]) for k in range(4)]

    def kernel_us(fn, reps=20):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps

    us_dg = kernel_us(lambda: sv.diffusion_exp_gradient(gt, lam, x, dg))
    us_dc = kernel_us(lambda: sv.coef_gradient(lam, x, dcoef))
    frac = lambda nb, us: round(nb / (us * 1e-6) / 1e9 / peak, 3)
    return {"workload": "1 part 128^3, 7-point harmonic-mean diffusion, kappa = exp(g), seed 4",
            "unknowns": N, "precision": "fp64",
            "setup_ms": round(t[0], 3), "forward_solve_ms": round(t[1], 3),
            "adjoint_solve_ms": round(t[2], 3), "gradient_ms": round(t[3], 3),
            "forward_iterations": st_f.iterations, "adjoint_iterations": st_a.iterations,
            "mdof_s": round(N / (sum(t) * 1e-3) / 1e6, 3),
            "k_diffusion_exp_gradient": {"us": round(us_dg, 2), "frac_hbm": frac(32 * N, us_dg)},
            "k_coef_gradient": {"us": round(us_dc, 2), "frac_hbm": frac(72 * N, us_dc)}}


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def end_to_end(S, prob, dev, stream, args):
    import torch
    N = prob.n
    b_pin = torch.from_numpy(prob.b[0].copy()).pin_memory()
    x_pin = torch.zeros(N, dtype=torch.float64).pin_memory()
    coef_pin = [[None if np.isscalar(c) else torch.from_numpy(np.ascontiguousarray(c).ravel()).pin_memory()
                 for c in part] for part in prob.coef]
    h2d = 8 * N + sum(t.numel() * 8 for part in coef_pin for t in part if t is not None) \
        + prob.nnz_u * (8 + 4 * 10)
    d2h = 8 * N

    def step():
        grid = S.Grid(prob.ndim, prob.boxes)
        A = S.Matrix(grid, prob.offsets)
        for p, part in enumerate(prob.coef):
            for e, c in enumerate(part):
                if coef_pin[p][e] is None:
                    A.set_constant(p, e, float(c))
                else:
                    A.set_box_values(p, e, coef_pin[p][e].numpy())
        A.add_couplings(prob.u_part, prob.u_idx, prob.u_dir, prob.u_nbor_part, prob.u_nbor_idx,
                        prob.u_val)
        A.assemble(stream)
        sv = S.Solver(precision=1, flexible=1, tol=1e-8, max_iter=500)
        sv.setup(A, stream)
        sv.solve_host(b_pin.numpy(), x_pin.numpy(), stream=stream, stats=False)
        return sv

    for _ in range(max(1, min(args.warmup, 2))):
        step()
    reps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    return {"value": round(N / dt / 1e6, 3), "unit": "MDOF/s", "ms_per_step": round(dt * 1e3, 3),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "includes": "grid+matrix creation from pinned host arrays, assemble, setup, solve, x read-back"}


def cpu_baseline(prob, sample_iters=2):
    """The oracle on the host: full setup plus the first `sample_iters` PCG
    iterations timed, extrapolated by the oracle's own iteration count."""
    from oracle import ssamg as O
    t0 = time.perf_counter()
    h = O.setup(prob)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.pcg(h, prob.b[0], max_iter=sample_iters)
    t_it = (time.perf_counter() - t0) / sample_iters
    iters = O.pcg(h, prob.b[0]).iterations
    total = t_setup + iters * t_it
    return {"value": round(prob.n / total / 1e6, 5), "unit": "MDOF/s", "cores": 1, "kind": "oracle",
            "sample": f"full setup + {sample_iters} of {iters} PCG iterations timed, extrapolated",
            "setup_s": round(t_setup, 3), "s_per_iteration": round(t_it, 4),
            "host": host_info()}


def host_info():
    try:
        import platform
        return {"nproc": os.cpu_count(), "machine": platform.machine()}
    except Exception:
        return {}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import ssamg as O
    prob = P.config(1)
    N = prob.n
    # the oracle's own iteration count (one full solve, untimed)
    h = O.setup(prob)
    iters = O.pcg(h, prob.b[0]).iterations
    sample_iters = 2
    for _ in range(args.warmup):
        O.vcycle(h, prob.b[0])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        h = O.setup(prob)
        t_setup = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.pcg(h, prob.b[0], max_iter=sample_iters)
        t_it = (time.perf_counter() - t0) / sample_iters
        times.append(t_setup + iters * t_it)
    step_s = statistics.median(times)
    v = N / step_s / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "MDOF/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(step_s * 1e3, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "unknowns": N, "tol": 1e-8, "parallelism": "cpu"},
        "cpu_baseline": {"value": round(v, 5), "unit": "MDOF/s", "cores": 1, "kind": "oracle",
                         "sample": f"per step: full setup + {sample_iters} of {iters} PCG iterations, extrapolated"},
        "e2e": {"value": round(v, 5), "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """A fixed case sized for ncu captures (inputs larger than L2, a few GB on
    the device at most)."""
    import torch

    from paper_2205_14273_gb300 import ssamg as S
    rng = P.SplitMix64(5)
    a = rng.log_uniform(6, 1e-3, 1.0).reshape(2, 3)
    prob = P.chain_aniso([200, 200], a, rng, 1)
    grid, A = S.matrix_from_problem(prob)
    sv = S.Solver(precision=1, flexible=1)
    sv.setup(A)
    b = torch.as_tensor(prob.b[0], device="cuda")
    z = torch.zeros_like(b)
    for _ in range(3):
        sv.precondition(b, z)
    # and three iterations of the flexible PCG (the cycle's PCG-side kernels)
    sv3 = S.Solver(precision=1, flexible=1, max_iter=3)
    sv3.setup(A)
    sv3.solve(b, z, allow_not_converged=True)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "cells": prob.n,
                      "levels": sv.num_levels()}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the solve kernels directly (profilers cannot see kernel "
                         "nodes of graphs with conditional nodes)")
    ap.add_argument("--only", choices=["fp32_cycle", "fp64"], default=None)
    ap.add_argument("--profile-case", choices=["level0-16M"], default=None,
                    help="run a fixed small case for profiler captures instead of the bench: "
                         "level0-16M = two chained 200^3 parts (16M cells, constant anisotropic "
                         "7-point off-diagonals, per-cell diagonal), FP32 cycle, setup, "
                         "three V-cycles and three flexible PCG iterations")
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="skip the 256^3 27-point and 64-problem batched measurements")
    ap.add_argument("--autotune", action="store_true",
                    help="run the tile autotuner on the main workload's solvers after the "
                         "warm-up (the timed set-ups then use the tuned tile table)")
    ap.add_argument("--levels", action="store_true",
                    help="also write, to stderr, each cycle kernel's time per level "
                         "(CUDA-graph replays of that launch alone)")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
