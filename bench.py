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

# the oracle's BLAS/OpenMP threads: 1 unless --cpu-threads asks otherwise
# (set before numpy is imported)
_THREADS = sys.argv[sys.argv.index("--cpu-threads") + 1] if "--cpu-threads" in sys.argv[:-1] else "1"
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, _THREADS)

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import problems as P  # noqa: E402

METRIC = "SSAMG-PCG setup+solve ms, MDOF/s to 1e-8 rel. res., FP32-cycle vs FP64; %HBM"
WORKLOAD = "8 parts x 64^3 (2x2x2 layout), 7-pt anisotropic diffusion, seed 1"
L2_BYTES = 129 * 2 ** 20
# FP64 peak of one GB300: 152 SMs x 2 FP64 FMA per clock per SM x 2 flops x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP64-pipe instructions per cell of dL/dg (exp(g), then six faces with a
# division each), counted by ncu on the 128^3 case
FP64_INSTS_PER_CELL_DG = 15 + 102


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
    ws, rank, local = dist_env()
    # the oracle beside the GPU: started before the first CUDA call
    beside = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        jobs = ["bench"] + ([] if args.no_extra_workloads else
                            ["laplace32", "diffusion128", "batched_subset", "samr128",
                             "three_point160", "multibox96"])
        beside = OracleBeside(jobs)

    import torch
    import torch.distributed as dist

    from paper_2205_14273_gb300 import ssamg as S

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
    xs = {}
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
        xs[name] = x.cpu().numpy()
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
        tl = sv.tail_levels()
        results[name]["coarse_transition"] = {"first_level": tl[0], "levels": tl[1]}
        if table is not None:
            results[name]["tile_table"] = tile_summary(table)

    if args.levels:
        for name, sv in solvers.items():
            level_table(sv, name, stream)

    # ---- roofline of the cycle's operations (all levels, all template instances)
    peak = read_peaks().get("hbm_gbs", 6800.0)
    roof = cycle_roofline(S, solvers.get("fp32_cycle", next(iter(solvers.values()))), prob, stream, peak)

    # ---- per-kernel HBM fractions on the large levels, and the other
    # full-size workloads
    hbm = hbm_by_level(solvers.get("fp32_cycle", next(iter(solvers.values()))),
                       "8 parts x 64^3", stream, peak)
    extra = None if args.no_extra_workloads else extra_workloads(S, stream, peak, args)

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
    if beside is None and extra is not None:
        strip_private(extra)
    if beside is not None:
        got = beside.result()
        if got is None:
            line["cpu_baseline"] = {"unavailable": "the oracle process did not finish"}
            if extra is not None:
                strip_private(extra)
        else:
            meta, arrays = got
            jb = meta["jobs"]["bench"]
            tot = jb["setup_s"] + jb["solve_s"]
            line["cpu_baseline"] = {
                "value": round(N / tot / 1e6, 5), "unit": "MDOF/s", "cores": 1, "kind": "oracle",
                "sample": f"one full oracle setup + PCG to 1e-8 ({jb['iterations']} iterations) "
                          f"of the whole workload, in a separate process beside the GPU run",
                "setup_s": round(jb["setup_s"], 3), "solve_s": round(jb["solve_s"], 3),
                "host": meta["host"]}
            # the error of each GPU result against the FP64 oracle's solution
            xo = arrays["bench:x"]
            for name in xs:
                line[name]["err_vs_oracle"] = fmt(rel_err(xs[name], xo))
            line["err_vs_oracle"] = {name: fmt(rel_err(xs[name], xo)) for name in xs}
            line["err_vs_oracle"]["oracle_iterations"] = jb["iterations"]
            if extra is not None:
                oracle_errors(extra, meta, arrays)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def cycle_roofline(S, sv, prob, stream, peak):
    """Roofline of the V-cycle's operations, each summed over the levels it
    runs on and over all its kernel instances (cell tiles, bricks, the
    precision's template): residual, post-relaxation (on level 0 the last
    relaxation as the PCG runs it, with the FP64 z and dot partials),
    restriction (with the coarse level's pre-relaxation and its U x rows),
    prolongation (with U x rows), level 0's pre-relaxation, and the coarse-
    level transition's cluster kernel (levels from its first on).  Each
    launch is timed alone (CUDA-graph replays on the solver's own buffers,
    CUDA events on the launching stream); achieved = algorithmic bytes / that
    time.  The operation with the largest summed time is the headline.

    Algorithmic bytes per level (FP32 cycle, w = 4; sc = stored per-cell
    coefficients of the level, nr/nnz its coupling rows and entries):
    residual w (sc + 3 N) + 4 nr; post-relaxation w (sc + 4 N) + 4 nr (level
    0: + 8 N FP64 r in, 8 N FP64 z out, 16 N FP64 zprev in/out);
    restriction w N_l + w N_{l+1} + 2 w (N_l - N_{l+1}) (+ 2 w N_{l+1} +
    12 nr + 44 nnz of the next level when it pre-relaxes there); prolongation
    8 N_l + 4 N_{l+1} + 8 (N_l - N_{l+1}) + 12 nr + 36 nnz; pre-relaxation
    (level 0) 8 N (FP64 r in) + 2 w N + 12 nr + 12 nnz."""
    L = sv.num_levels()
    sizes = [sv.level_sizes(l) for l in range(L)]
    first, ntail = sv.tail_levels()
    lt = first if ntail else L - 1        # levels below lt run per-level kernels
    w = 4
    sc = [sv.stored_coefficients(l) for l in range(L)]

    def b_res(l):
        N, nr, _ = sizes[l]
        return w * (sc[l] + 3 * N) + 4 * nr

    def b_relax(l):
        N, nr, _ = sizes[l]
        return w * (sc[l] + 4 * N) + 4 * nr + (32 * N if l == 0 else 0)

    def b_restrict(l):
        N = sizes[l][0]
        Nc, nrc, nnzc = sizes[l + 1]
        pre = 2 * w * Nc + 12 * nrc + 44 * nnzc if l + 1 < lt else 0
        return w * N + w * Nc + 2 * w * (N - Nc) + pre

    def b_prolong(l):
        N, nr, nnz = sizes[l]
        Nc = sizes[l + 1][0]
        return 8 * N + 4 * Nc + 8 * (N - Nc) + 12 * nr + 36 * nnz

    def b_pre(l):
        N, nr, nnz = sizes[l]
        return 8 * N + 2 * w * N + 12 * nr + 12 * nnz

    ops = {
        "residual": (lambda l: 0, b_res, range(lt)),
        "post_relaxation": (lambda l: 9 if l == 0 else 1, b_relax, range(lt)),
        "restriction": (lambda l: 3, b_restrict, range(lt)),
        "prolongation": (lambda l: 4, b_prolong, range(lt)),
        "pre_relaxation_level0": (lambda l: 2, b_pre, range(1)),
    }
    by_op = {}
    for name, (kid, nbytes, levels) in ops.items():
        us = [sv.time_kernel(kid(l), l, 50, stream) for l in levels]
        tb = sum(nbytes(l) for l in levels)
        tus = sum(us)
        gbs = tb / (tus * 1e-6) / 1e9
        by_op[name] = {"levels": len(us), "us": round(tus, 2), "bytes": int(tb),
                       "achieved_gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                       "us_per_level": [round(u, 2) for u in us]}
    if ntail:
        by_op["coarse_transition_cluster"] = {
            "levels": ntail, "first_level": first, "us": round(sv.time_kernel(10, 0, 50, stream), 2),
            "bound": "latency (cluster barriers and remote shared-memory round trips)"}
    cycle_us = sv.time_kernel(5, 0, 20, stream)
    top = max((k for k in ops), key=lambda k: by_op[k]["us"])
    t = by_op[top]
    nl = t["levels"]
    out = {
        "kernel": f"{top} of the FP32 V-cycle, all its kernel instances, levels 0..{lt - 1} "
                  f"(the operation with the largest summed launch time)",
        "bound": "hbm", "achieved": t["achieved_gbs"], "peak": peak, "unit": "GB/s",
        "frac": t["frac"], "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
        "traffic": None,
        "traffic_note": "the 2M-cell levels' data stays in the 129 MB L2 between launches, so "
                        "DRAM counters read below the algorithmic bytes; the HBM-resident "
                        "case is in other_workloads and profiles/",
        "bytes_per_launch": int(t["bytes"] / max(nl, 1)), "us_per_launch": round(t["us"] / max(nl, 1), 3),
        "v_cycle_us": round(cycle_us, 1),
        "by_operation": by_op,
    }
    # the PCG's FP64 level-0 operator apply + dot (bound by the FP64 pipe)
    us_spmv = sv.time_kernel(6, 0, 50, stream)
    N0 = sizes[0][0]
    flops = 2 * 8 * N0 + 2 * prob.nnz_u
    out["fp64_level0_operator"] = {
        "kernel": "k7b_spmv_dot (q = A p and p.q, FP64, level 0 bricks)",
        "bound": "alu", "unit": "TFLOP/s",
        "achieved": round(flops / (us_spmv * 1e-6) / 1e12, 4),
        "peak": FP64_PEAK_TFLOPS, "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x 2.07 GHz",
        "frac": round(flops / (us_spmv * 1e-6) / (FP64_PEAK_TFLOPS * 1e12), 4),
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


def hbm_by_level(sv, workload, stream, peak, min_cells=1 << 20, nrhs=1):
    """Per-kernel HBM throughput of the FP32 cycle on the levels of at least
    2^20 cells: algorithmic bytes (each input and output once; w = 4) / the
    kernel's CUDA-graph launch time (50 replayed launches on the solver's own
    buffers), against the measured copy bandwidth.  Launches moving less than
    ~3/4 of L2 are flagged l2_resident.  With nrhs > 1 (after a batch solve of
    that many right-hand sides together), the residual and relaxation of
    cell-tile levels are also timed as the solve runs them, every right-hand
    side in one launch: the coefficients counted once, the vectors nrhs
    times."""
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
        if nrhs > 1 and not sv.level_tile(l)[1]:
            for k, kid, nb in (("residual_rhs_together", 11, w * (sc + 3 * N * nrhs)),
                               ("relax_rhs_together", 12, w * (sc + 4 * N * nrhs))):
                us = sv.time_kernel(kid, l, 50, stream)
                gbs = nb / (us * 1e-6) / 1e9
                row[k] = {"rhs": nrhs, "us": round(us, 2), "us_per_rhs": round(us / nrhs, 2),
                          "gbs": round(gbs, 1), "frac": round(gbs / peak, 3)}
        rows.append(row)
    return {"workload": workload, "peak_gbs": peak, "levels": rows}


def tile_summary(table):
    """Non-default entries of a tile table: size class -> form."""
    return {f"2^{c}": (f"{t & 7} cells/thread" + (" + bricks" if t & 8 else ""))
            for c, t in enumerate(table) if t}


def timed_steps(stream, nsteps, setup, solve, local=0):
    """nsteps setup + solve steps, each bracketed by CUDA events on `stream`,
    with nvidia-smi clocks sampled meanwhile; medians (ms) and the clocks."""
    import torch
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(nsteps)]
    ck = ClockSampler(local)
    torch.cuda.synchronize()
    ck.start()
    last = None
    for e in ev:
        e[0].record(stream)
        setup()
        e[1].record(stream)
        last = solve()
        e[2].record(stream)
    torch.cuda.synchronize()
    clocks = ck.stop()
    su = [e[0].elapsed_time(e[1]) for e in ev]
    so = [e[1].elapsed_time(e[2]) for e in ev]
    return statistics.median(su), statistics.median(so), clocks, last


def golden_var27():
    path = os.path.join(ROOT, "tests", "golden", "var27_256_oracle.json")
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return None


def extra_workloads(S, stream, peak, args):
    """The other full-size workloads: 32^3 Laplacian (FP64; latency),
    256^3 27-point, the 64-problem batch, the 128^3 differentiation
    workload and the paper's test cases 3 (three-point intersection,
    3 x 160^3) and 4 (SAMR, 2 x 128^3): setup and solve times (median of 5
    steps after a warm-up,
    clocks sampled), per-kernel HBM fractions of the large levels, and each
    solution's error against the FP64 oracle (256^3: on the oracle's stored
    samples; batch: on its eight smallest problems; the rest in full)."""
    import torch
    out = {}
    nst = 5
    # ---- 32^3 Laplacian, plain FP64 (reported as latency)
    prob = P.config(0)
    grid, A = S.matrix_from_problem(prob)
    b = torch.as_tensor(prob.b[0], device="cuda")
    x = torch.zeros_like(b)
    sv = S.Solver(tol=1e-8, max_iter=500)
    sv.setup(A)
    st = sv.solve(b, x)
    su, so, ck, _ = timed_steps(stream, 10, lambda: sv.setup(A), lambda: sv.solve_nostats(b, x))
    out["laplace_32"] = {"workload": "1 part 32^3, 7-point Laplacian, FP64 cycle, seed 0",
                         "unknowns": prob.n, "setup_ms": round(su, 3), "solve_ms": round(so, 3),
                         "latency_ms": round(su + so, 3), "iterations": st.iterations,
                         "mdof_s": round(prob.n / ((su + so) * 1e-3) / 1e6, 3), "steps": 10,
                         "clocks": ck, "_x": x.cpu().numpy()}
    del A, grid, sv
    # ---- 256^3 27-point
    prob = P.config(2)
    grid, A = S.matrix_from_problem(prob)
    b = torch.as_tensor(prob.b[0], device="cuda")
    res = {"workload": "1 part 256^3, 27-point variable coefficients, seed 2",
           "unknowns": prob.n}
    gold = golden_var27()
    for prec, name in ((1, "fp32_cycle"), (0, "fp64")):
        sv = S.Solver(precision=prec, flexible=prec, tol=1e-8, max_iter=500)
        sv.setup(A)
        x = torch.zeros_like(b)
        st = sv.solve(b, x)
        su, so, ck, _ = timed_steps(stream, nst, lambda: sv.setup(A), lambda: sv.solve_nostats(b, x))
        res[name] = {"setup_ms": round(su, 3), "solve_ms": round(so, 3),
                     "iterations": st.iterations, "true_rel_res": fmt(st.true_rel_res),
                     "levels": st.num_levels, "steps": nst, "clocks": ck,
                     "mdof_s": round(prob.n / ((su + so) * 1e-3) / 1e6, 3)}
        if gold is not None:
            cells = np.array(gold["pcg"]["cells"])
            xo = np.array(gold["pcg"]["x"])
            xg = x.cpu().numpy()[cells]
            res[name]["err_vs_oracle"] = {
                "sampled_rel_err": fmt(rel_err(xg, xo)), "samples": len(cells),
                "norm_ratio": fmt(float(x.norm()) / gold["pcg"]["x_norm"]),
                "oracle_iterations": gold["pcg"]["iterations"]}
        if prec == 1:
            res["hbm"] = hbm_by_level(sv, res["workload"], stream, peak)
        del sv
    out["var27_256"] = res
    del A, grid
    # ---- 64 problems x 4 right-hand sides
    probs = P.config(3)
    mats = [S.matrix_from_problem(p) for p in probs]
    nrhs = probs[0].b.shape[0]
    sel = batched_subset(probs)
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
        B.solve(bb, xx, nrhs)
        su_u, so_u, _, _ = timed_steps(stream, 1, B.setup, lambda: B.solve(bb, xx, nrhs))
        t0 = time.perf_counter()
        table = B.autotune(reps=10)
        tune_s = time.perf_counter() - t0
        B.solve(bb, xx, nrhs)
        su, so, ck, st = timed_steps(stream, nst, B.setup, lambda: B.solve(bb, xx, nrhs))
        its = [s_.iterations for row in st for s_ in row]
        res["unknowns"] = off[-1]
        xh = xx.cpu().numpy()
        res[name] = {"setup_ms": round(su, 3), "solve_ms": round(so, 3), "steps": nst, "clocks": ck,
                     "tile_table": tile_summary(table), "autotune_s": round(tune_s, 2),
                     "builtin_tiles": {"setup_ms": round(su_u, 3), "solve_ms": round(so_u, 3)},
                     "iterations_max": max(its), "iterations_mean": round(float(np.mean(its)), 2),
                     "worst_true_rel_res": fmt(max(s_.true_rel_res for row in st for s_ in row)),
                     "levels": st[0][0].num_levels,
                     "mdof_s": round(off[-1] * nrhs / ((su + so) * 1e-3) / 1e6, 3),
                     "_x": {f"{k}_{j}": xh[j, off[k]:off[k + 1]].copy() for k in sel for j in range(nrhs)}}
        if prec == 1:
            res["hbm"] = hbm_by_level(B.solver(), res["workload"], stream, peak, nrhs=nrhs)
            # the same batch and tile table with the right-hand sides one
            # after another (each its own PCG loop inside the one graph)
            B2 = S.Batch([A for _, A in mats], precision=prec, flexible=prec, tol=1e-8,
                         max_iter=500, rhs_together=0)
            B2.solver().set_tile_table(table)
            B2.setup()
            x2 = torch.zeros_like(bb)
            B2.solve(bb, x2, nrhs)
            su2, so2, _, st2 = timed_steps(stream, nst, B2.setup, lambda: B2.solve(bb, x2, nrhs))
            res[name]["rhs_one_after_another"] = {
                "setup_ms": round(su2, 3), "solve_ms": round(so2, 3), "steps": nst,
                "solutions_bitwise_equal": bool(torch.equal(xx, x2)),
                "mdof_s": round(off[-1] * nrhs / ((su2 + so2) * 1e-3) / 1e6, 3)}
            del B2, x2
        del B
    out["batched_64"] = res
    out["diffusion_128"] = differentiation_workload(S, stream, peak)
    # ---- Section 4 test cases 3 (non-Cartesian index maps) and 4 (SAMR)
    for key, k, text in (("three_point_160", 5, "3 parts 160^3 around a common k edge, rotated "
                                                "index maps (test case 3), seed 5"),
                         ("samr_128", 6, "2 parts 128^3: coarse grid with ghost unknowns and a "
                                         "patch refined by 2 (test case 4), seed 6"),
                         ("multibox_96", 7, "an L-shaped part of two boxes (3 x 96^3 cells, held "
                                            "over its 192 x 192 x 96 bounding box) around a 96^3 "
                                            "part, seed 7")):
        prob = P.config(k)
        grid, A = S.matrix_from_problem(prob)
        b = torch.as_tensor(prob.b[0], device="cuda")
        res = {"workload": text, "unknowns": prob.n}
        for prec, name in ((1, "fp32_cycle"), (0, "fp64")):
            sv = S.Solver(precision=prec, flexible=prec, tol=1e-8, max_iter=500)
            sv.setup(A)
            x = torch.zeros_like(b)
            st = sv.solve(b, x)
            su, so, ck, _ = timed_steps(stream, nst, lambda: sv.setup(A), lambda: sv.solve_nostats(b, x))
            res[name] = {"setup_ms": round(su, 3), "solve_ms": round(so, 3),
                         "iterations": st.iterations, "true_rel_res": fmt(st.true_rel_res),
                         "levels": st.num_levels, "steps": nst, "clocks": ck,
                         "mdof_s": round(prob.n / ((su + so) * 1e-3) / 1e6, 3),
                         "_x": x.cpu().numpy()}
            del sv
        out[key] = res
        del A, grid
    return out


def oracle_errors(extra, meta, arrays):
    """Fills err_vs_oracle of the other workloads from the oracle run beside
    (and drops the solution vectors kept for it)."""
    jobs = meta["jobs"]
    lap = extra.get("laplace_32")
    if lap is not None:
        x = lap.pop("_x")
        if "laplace32" in jobs:
            lap["err_vs_oracle"] = fmt(rel_err(x, arrays["laplace32:x"]))
            lap["oracle_iterations"] = jobs["laplace32"]["iterations"]
    bat = extra.get("batched_64")
    if bat is not None:
        for name in ("fp32_cycle", "fp64"):
            xs = bat[name].pop("_x", {})
            if "batched_subset" in jobs and xs:
                errs = [rel_err(v, arrays[f"batched_subset:x:{k}"]) for k, v in xs.items()]
                bat[name]["err_vs_oracle"] = {"max_rel_err": fmt(max(errs)), "instances": len(errs),
                                              "problems": jobs["batched_subset"]["problems"]}
    for key, job in (("three_point_160", "three_point160"), ("samr_128", "samr128"),
                     ("multibox_96", "multibox96")):
        w = extra.get(key)
        if w is None:
            continue
        for name in ("fp32_cycle", "fp64"):
            x = w[name].pop("_x", None)
            if job in jobs and x is not None:
                w[name]["err_vs_oracle"] = fmt(rel_err(x, arrays[f"{job}:x"]))
        if job in jobs:
            w["oracle_iterations"] = jobs[job]["iterations"]
    dif = extra.get("diffusion_128")
    if dif is not None:
        x, dg = dif.pop("_x"), dif.pop("_dg")
        if "diffusion128" in jobs:
            dif["err_vs_oracle"] = {"x": fmt(rel_err(x, arrays["diffusion128:x"])),
                                    "dL_dg": fmt(rel_err(dg, arrays["diffusion128:dg"])),
                                    "oracle_iterations": [jobs["diffusion128"]["iterations"],
                                                          jobs["diffusion128"]["adjoint_iterations"]]}


def strip_private(extra):
    """Drops the solution vectors kept for the oracle comparison (no oracle run)."""
    for w in extra.values():
        if isinstance(w, dict):
            for k in [k for k in w if k.startswith("_")]:
                w.pop(k)
            for v in w.values():
                if isinstance(v, dict):
                    for k in [k for k in v if k.startswith("_")]:
                        v.pop(k)


def differentiation_workload(S, stream, peak):
    """The differentiation form at full size (128^3, kappa = exp(g), FP64):
    setup, forward solve, adjoint solve A lambda = x - x_t on the same
    hierarchy, and dL/dg, each timed with CUDA events (median of 5 steps after
    a warm-up step); the gradient kernels' HBM fractions
    (k_diffusion_exp_gradient: g, lambda, x in and dL/dg out, 32 B per cell;
    k_coef_gradient: lambda and x in, the 7 entries' dL/da out, 72 B per
    cell)."""
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
    ts = []
    for _ in range(5):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        st_f, st_a = step(ev)
        torch.cuda.synchronize()
        ts.append([ev[k].elapsed_time(ev[k + 1]) for k in range(4)])
    t = [statistics.median(c) for c in zip(*ts)]

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
            "unknowns": N, "precision": "fp64", "steps": 5,
            "setup_ms": round(t[0], 3), "forward_solve_ms": round(t[1], 3),
            "adjoint_solve_ms": round(t[2], 3), "gradient_ms": round(t[3], 3),
            "forward_iterations": st_f.iterations, "adjoint_iterations": st_a.iterations,
            "mdof_s": round(N / (sum(t) * 1e-3) / 1e6, 3),
            "k_diffusion_exp_gradient": {
                "us": round(us_dg, 2), "frac_hbm": frac(32 * N, us_dg),
                # bound by the FP64 pipe: FP64-pipe instructions per cell
                # counted by ncu (15 in k_exp, 102 in the gradient kernel)
                # against 2 per SM per clock (152 SMs, 2.07 GHz)
                "bound": "fp64",
                "fp64_pipe_insts_per_cell": FP64_INSTS_PER_CELL_DG,
                "frac_fp64_pipe": round(FP64_INSTS_PER_CELL_DG * N / (us_dg * 1e-6)
                                        / (FP64_PEAK_TFLOPS * 1e12 / 2), 3)},
            "k_coef_gradient": {"us": round(us_dc, 2), "frac_hbm": frac(72 * N, us_dc)},
            "_x": x.cpu().numpy(), "_dg": dg.cpu().numpy()}


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


# ---------------------------------------------------------------------------
# The CPU oracle beside the GPU (cpu_baseline, the errors against the FP64
# oracle, the reference arm).  Every oracle run is a full setup and a full
# PCG solve to the workload's tolerance, timed as it stands (never tuned).
# ---------------------------------------------------------------------------
def host_info():
    info = {"nproc": os.cpu_count()}
    try:
        import platform
        info["machine"] = platform.machine()
    except Exception:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                info["cpu_model"] = line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        cfg = np.show_config(mode="dicts")
        info["blas"] = cfg["Build Dependencies"]["blas"]["name"]
    except Exception:
        pass
    info["numpy"] = np.__version__
    info["threads_env"] = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    return info


def batched_subset(probs, k=8):
    """The k problems of the batched workload with the fewest cells."""
    return sorted(range(len(probs)), key=lambda i: (probs[i].n, i))[:k]


def oracle_run(job):
    """One timed oracle job (full setup and PCG to 1e-8); returns its timings
    and the solution vectors (numpy)."""
    from oracle import ssamg as O
    out = {}
    if job in ("bench", "laplace32"):
        prob = P.config(1 if job == "bench" else 0)
        t0 = time.perf_counter()
        h = O.setup(prob)
        t1 = time.perf_counter()
        r = O.pcg(h, prob.b[0], tol=1e-8, max_iter=500)
        t2 = time.perf_counter()
        out = {"setup_s": t1 - t0, "solve_s": t2 - t1, "iterations": r.iterations,
               "true_rel_res": r.true_rel_res, "unknowns": prob.n, "x": r.x}
    elif job == "diffusion128":
        prob = P.config(4)
        t0 = time.perf_counter()
        h = O.setup(prob)
        t1 = time.perf_counter()
        r = O.pcg(h, prob.b[0], tol=1e-8, max_iter=500)
        t2 = time.perf_counter()
        ra = O.pcg(h, r.x - prob.extra["x_t"], tol=1e-8, max_iter=500)
        t3 = time.perf_counter()
        dg = O.diffusion_exp_gradient(prob.extra["g"], ra.x, r.x).reshape(-1)
        t4 = time.perf_counter()
        out = {"setup_s": t1 - t0, "solve_s": t2 - t1, "adjoint_s": t3 - t2, "gradient_s": t4 - t3,
               "iterations": r.iterations, "adjoint_iterations": ra.iterations,
               "unknowns": prob.n, "x": r.x, "dg": dg}
    elif job in ("three_point160", "samr128", "multibox96"):
        prob = P.config({"three_point160": 5, "samr128": 6, "multibox96": 7}[job])
        t0 = time.perf_counter()
        h = O.setup(prob)
        t1 = time.perf_counter()
        r = O.pcg(h, prob.b[0], tol=1e-8, max_iter=500)
        t2 = time.perf_counter()
        out = {"setup_s": t1 - t0, "solve_s": t2 - t1, "iterations": r.iterations,
               "true_rel_res": r.true_rel_res, "unknowns": prob.n, "x": r.x}
    elif job == "batched_subset":
        probs = P.config(3)
        sel = batched_subset(probs)
        xs, its = {}, []
        t0 = time.perf_counter()
        n = 0
        for k in sel:
            h = O.setup(probs[k])
            for j in range(probs[k].b.shape[0]):
                r = O.pcg(h, probs[k].b[j], tol=1e-8, max_iter=500)
                xs[f"{k}_{j}"] = r.x
                its.append(r.iterations)
                n += probs[k].n
        out = {"problems": sel, "seconds": time.perf_counter() - t0, "unknowns_x_rhs": n,
               "iterations": its, "x": xs}
    return out


def oracle_worker(out_path, jobs):
    """Spawned process: the oracle jobs in turn; timings to JSON, vectors to
    an .npz beside it."""
    res, arrays = {}, {}
    for job in jobs:
        r = oracle_run(job)
        for key in list(r):
            v = r[key]
            if isinstance(v, np.ndarray):
                arrays[f"{job}:{key}"] = r.pop(key)
            elif isinstance(v, dict):
                for kk, vv in r.pop(key).items():
                    arrays[f"{job}:{key}:{kk}"] = vv
        res[job] = r
    np.savez(out_path + ".npz", **arrays)
    with open(out_path + ".json", "w") as f:
        json.dump({"jobs": res, "host": host_info()}, f)


class OracleBeside:
    """The oracle jobs in a spawned process (started before the first GPU call,
    so that no CUDA state is inherited), running while the GPU is timed."""

    def __init__(self, jobs):
        import multiprocessing as mp
        self.dir = tempfile.mkdtemp(prefix="ssamg_oracle_")
        self.path = os.path.join(self.dir, "oracle")
        self.proc = mp.get_context("spawn").Process(target=oracle_worker, args=(self.path, jobs))
        self.proc.start()

    def result(self, timeout=900):
        self.proc.join(timeout)
        if self.proc.is_alive():
            self.proc.terminate()
            return None
        if self.proc.exitcode != 0 or not os.path.exists(self.path + ".json"):
            return None
        with open(self.path + ".json") as f:
            meta = json.load(f)
        arrays = dict(np.load(self.path + ".npz"))
        return meta, arrays


def rel_err(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_reference(args):
    """The reference arm: the CPU oracle (there is no reference code) on this
    workload, timed as it stands on the host cores: each step is one full
    setup and one full PCG solve to 1e-8 of the 8 x 64^3 workload.  A step
    takes ~20 s, so the arm runs min(steps, 3) steps after one untimed small
    warm-up run and reports the median; steps/warmup requested are recorded."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import ssamg as O
    prob = P.config(1)
    N = prob.n
    small = P.config(1, small=True)
    O.pcg(O.setup(small), small.b[0], tol=1e-8)
    nsteps = max(1, min(args.steps, 3))
    times, its = [], []
    for _ in range(nsteps):
        t0 = time.perf_counter()
        h = O.setup(prob)
        r = O.pcg(h, prob.b[0], tol=1e-8, max_iter=500)
        times.append(time.perf_counter() - t0)
        its.append(r.iterations)
    step_s = statistics.median(times)
    v = N / step_s / 1e6
    host = host_info()
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "MDOF/s",
        "n_gpus": ws, "steps": nsteps, "warmup": 1, "steps_requested": args.steps,
        "warmup_requested": args.warmup,
        "ms_per_step": round(step_s * 1e3, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "unknowns": N, "tol": 1e-8, "parallelism": "cpu"},
        "cpu_baseline": {"value": round(v, 5), "unit": "MDOF/s", "cores": 1, "kind": "oracle",
                         "sample": f"per step: one full oracle setup + PCG to 1e-8 "
                                   f"({its[0]} iterations) of the whole workload; "
                                   f"median of {nsteps} steps",
                         "host": host},
        "e2e": {"value": round(v, 5), "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_cpu_table(args):
    """Oracle timings for the five workloads (the benchmark's table): setup and
    solve seconds, iterations, MDOF/s, with the threads given by
    --cpu-threads (BLAS/OpenMP variables; the oracle's numpy array arithmetic
    runs on one core either way).  Median of 3 runs for the 32^3 and 8 x 64^3
    workloads, one run for the others; the batched workload on its eight
    smallest problems (all right-hand sides), scaled by unknowns."""
    out = {"threads": args.cpu_threads, "host": host_info(), "workloads": {}}
    for job, reps in (("laplace32", 3), ("bench", 3), ("diffusion128", 1), ("batched_subset", 1)):
        runs = [oracle_run(job) for _ in range(reps)]
        for r in runs:
            for k in list(r):
                if isinstance(r[k], (np.ndarray, dict)):
                    r.pop(k)
        if job == "batched_subset":
            r = runs[0]
            out["workloads"][job] = {"seconds": r["seconds"], "unknowns_x_rhs": r["unknowns_x_rhs"],
                                     "mdof_s": r["unknowns_x_rhs"] / r["seconds"] / 1e6,
                                     "iterations_max": max(r["iterations"]),
                                     "problems": r["problems"]}
            continue
        tot = [r["setup_s"] + r["solve_s"] + r.get("adjoint_s", 0) + r.get("gradient_s", 0) for r in runs]
        med = sorted(range(reps), key=lambda i: tot[i])[reps // 2]
        r = runs[med]
        r["total_s"] = tot[med]
        r["mdof_s"] = r["unknowns"] / tot[med] / 1e6
        r["runs"] = reps
        out["workloads"][job] = r
    if args.cpu_var27:
        from oracle import ssamg as O
        prob = P.config(2)
        t0 = time.perf_counter()
        h = O.setup(prob)
        t1 = time.perf_counter()
        r = O.pcg(h, prob.b[0], tol=1e-8, max_iter=500)
        t2 = time.perf_counter()
        out["workloads"]["var27_256"] = {"setup_s": t1 - t0, "solve_s": t2 - t1,
                                         "iterations": r.iterations, "unknowns": prob.n,
                                         "mdof_s": prob.n / (t2 - t0) / 1e6, "runs": 1}
    print(json.dumps(out), flush=True)


def run_profile_case(args):
    """A fixed case sized for ncu captures (inputs larger than L2, a few GB on
    the device at most)."""
    import torch

    from paper_2205_14273_gb300 import ssamg as S
    if args.profile_case == "diffusion-128":
        # the differentiation workload's gradient kernels (FP64, 128^3):
        # forward and adjoint solve, then dL/dg three times
        prob = P.config(4)
        grid, A = S.matrix_from_problem(prob)
        sv = S.Solver(tol=1e-8, max_iter=500, use_graph=0)
        sv.setup(A)
        b = torch.as_tensor(prob.b[0], device="cuda")
        x = torch.zeros_like(b)
        lam = torch.zeros_like(b)
        dg = torch.zeros_like(b)
        sv.solve(b, x)
        sv.adjoint_solve(x - torch.as_tensor(prob.extra["x_t"], device="cuda"), lam)
        g = torch.as_tensor(prob.extra["g"].reshape(-1), device="cuda")
        for _ in range(3):
            sv.diffusion_exp_gradient(g, lam, x, dg)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": args.profile_case, "cells": prob.n}))
        return
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
    ap.add_argument("--profile-case", choices=["level0-16M", "diffusion-128"], default=None,
                    help="run a fixed small case for profiler captures instead of the bench: "
                         "level0-16M = two chained 200^3 parts (16M cells, constant anisotropic "
                         "7-point off-diagonals, per-cell diagonal), FP32 cycle, setup, "
                         "three V-cycles and three flexible PCG iterations; diffusion-128 = the "
                         "128^3 differentiation workload, forward and adjoint solve, three "
                         "dL/dg evaluations")
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="skip the 256^3 27-point and 64-problem batched measurements")
    ap.add_argument("--autotune", action="store_true",
                    help="run the tile autotuner on the main workload's solvers after the "
                         "warm-up (the timed set-ups then use the tuned tile table)")
    ap.add_argument("--levels", action="store_true",
                    help="also write, to stderr, each cycle kernel's time per level "
                         "(CUDA-graph replays of that launch alone)")
    ap.add_argument("--cpu-table", action="store_true",
                    help="time the CPU oracle on the workloads (no GPU) and print one JSON line")
    ap.add_argument("--cpu-threads", type=int, default=1,
                    help="BLAS/OpenMP threads for --cpu-table")
    ap.add_argument("--cpu-var27", action="store_true",
                    help="with --cpu-table, also the 256^3 27-point workload (minutes)")
    args = ap.parse_args()
    if args.cpu_table:
        run_cpu_table(args)
        return
    if args.profile_case:
        run_profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
