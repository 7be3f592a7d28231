"""Parity at the workloads' full sizes, in the bench's launch configuration
(CUDA graph, programmatic dependent launch, default parameters).

* 8 parts x 64^3 (the bench workload): every level of the hierarchy against
  the oracle (1e-12 per level), one V-cycle (1e-12; FP32 cycle 5e-5), the PCG
  iteration count at 1e-8 against the oracle's (within one) and the true
  residual.
* 256^3 27-point variable coefficients: level-0 operator apply on sampled
  cells from the problem's own coefficients, level-0 P weights against the
  oracle, the level-1 operator against the oracle's P^T A P applied to a
  random vector (the Galerkin identity at full size), V-cycle symmetry, and
  the PCG residual in both precisions with the FP32 cycle's solution error
  against the FP64 one stated.
* 128^3 diffusion: dL/dg against central finite differences on the 32 probe
  cells (bound 2e-6 of the largest probed derivative: the noise floor of a
  difference quotient at 2M cells).
"""
import numpy as np
import pytest

import problems as P
from oracle import ssamg as O

import test_gpu_parity as G

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def S(ssamg_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ssamg_lib


@pytest.fixture(scope="module")
def bench_case():
    prob = P.config(1)
    return prob, O.setup(prob)


def test_bench_workload_hierarchy(S, bench_case):
    prob, h = bench_case
    _, _, sv = G.gpu_setup(S, prob)
    G.compare_hierarchy(S, prob, sv, h)


def test_bench_workload_vcycle(S, bench_case):
    prob, h = bench_case
    r = P.SplitMix64(29).uniform_pm1(prob.n)
    zr = O.vcycle(h, r)
    rt = torch.as_tensor(r, device="cuda")
    for prec, tol in ((0, G.OP_TOL), (1, 5e-5)):
        _, _, sv = G.gpu_setup(S, prob, precision=prec, flexible=prec)
        z = torch.zeros_like(rt)
        sv.precondition(rt, z)
        assert G.rel(z.cpu().numpy(), zr) <= tol, prec


def test_bench_workload_pcg(S, bench_case):
    prob, h = bench_case
    b = prob.b[0]
    ref = O.pcg(h, b, tol=1e-8)
    bt = torch.as_tensor(b, device="cuda")
    for prec in (0, 1):
        _, _, sv = G.gpu_setup(S, prob, precision=prec, flexible=prec, tol=1e-8, max_iter=500)
        x = torch.zeros_like(bt)
        st = sv.solve(bt, x)
        assert st.converged and st.true_rel_res <= 1.05e-8, prec
        assert abs(st.iterations - ref.iterations) <= 1, (prec, st.iterations, ref.iterations)


def _stencil_at(prob, cells, x):
    """(A x) at the given cells of a one-part problem, summed entry by entry
    from the problem's coefficient arrays (connections leaving the box
    dropped)."""
    (lo, hi), = prob.boxes
    n = [hi[d] - lo[d] + 1 for d in range(3)]
    i = cells % n[0]
    j = (cells // n[0]) % n[1]
    k = cells // (n[0] * n[1])
    out = np.zeros(len(cells))
    for e, o in enumerate(prob.offsets):
        c = prob.coef[0][e]
        a = np.full(len(cells), float(c)) if np.isscalar(c) else np.asarray(c).reshape(-1)[cells]
        ii, jj, kk = i + o[0], j + o[1], k + o[2]
        ok = (ii >= 0) & (ii < n[0]) & (jj >= 0) & (jj < n[1]) & (kk >= 0) & (kk < n[2])
        nb = np.where(ok, (kk * n[1] + jj) * n[0] + ii, 0)
        out += np.where(ok, a * x[nb], 0.0)
    return out


def test_var27_full_size(S):
    prob = P.config(2)
    N = prob.n
    gen = P.SplitMix64(31)
    x = gen.uniform_pm1(N)
    cells = gen.int_range(4096, 0, N - 1)
    # level-0 apply, sampled
    _, _, sv = G.gpu_setup(S, prob)
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    sv.level_matvec(0, torch.as_tensor(x, device="cuda"), y)
    ref = _stencil_at(prob, cells, x)
    got = y.cpu().numpy()[cells]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # level-0 coarsening decision and P, and the level-1 operator, against
    # the oracle's first coarsening step
    lev0 = O.level0_from_problem(prob)
    W0 = O.grid_spacings(O.coupling_sums(lev0), 3)
    boxes, dstars, omegas = O.coarsen_plan(W0, lev0.lo, lev0.hi, 3, 1, 2)
    lev0.dstar, lev0.omega = dstars[0], omegas[0]
    info = sv.part_info(0, 0)
    assert info["dstar"] == dstars[0][0]
    d = dstars[0][0]
    PW, PE = O.interpolation(lev0, 0, d)
    gW, gE = G.gpu_p(sv, 0, 0, info, lev0.shape(0))
    assert np.abs(gW - PW).max() <= G.OP_TOL and np.abs(gE - PE).max() <= G.OP_TOL
    lev0.PW, lev0.PE = [PW], [PE]
    nlo, nhi = boxes[1]
    coarse = O.Level(3, [np.array(v) for v in nlo], [np.array(v) for v in nhi], [None])
    lev0.P = O.prolongation_coo(lev0, coarse)
    n1 = sv.level_sizes(1)[0]
    yc = gen.uniform_pm1(n1)
    ref1 = O.restrict(lev0, O.matvec(lev0, O.prolong(lev0, yc)), n1)
    z1 = torch.zeros(n1, dtype=torch.float64, device="cuda")
    sv.level_matvec(1, torch.as_tensor(yc, device="cuda"), z1)
    assert G.rel(z1.cpu().numpy(), ref1) <= 1e-12
    # V-cycle symmetry <M r1, r2> = <r1, M r2>
    r1 = torch.as_tensor(gen.uniform_pm1(N), device="cuda")
    r2 = torch.as_tensor(gen.uniform_pm1(N), device="cuda")
    m1, m2 = torch.zeros_like(r1), torch.zeros_like(r2)
    sv.precondition(r1, m1)
    sv.precondition(r2, m2)
    a, b = float(torch.dot(m1, r2)), float(torch.dot(r1, m2))
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))
    # PCG in both precisions; the FP32 cycle's solution error against FP64
    bt = torch.as_tensor(prob.b[0], device="cuda")
    xs = {}
    for prec in (0, 1):
        _, _, s2 = G.gpu_setup(S, prob, precision=prec, flexible=prec, tol=1e-8, max_iter=500)
        xx = torch.zeros_like(bt)
        st = s2.solve(bt, xx)
        assert st.converged and st.true_rel_res <= 1.05e-8, prec
        xs[prec] = xx
    err = float((xs[1] - xs[0]).norm() / xs[0].norm())
    print(f"256^3 27-point: FP32-cycle solution vs FP64, relative 2-norm difference {err:.3e}")
    assert err <= 1e-4


def test_diffusion_full_size_gradient_fd(S):
    prob = P.config(4)
    g, xt, b = prob.extra["g"], prob.extra["x_t"], prob.b[0]
    # forward, adjoint and probe solves to 1e-15 (or the iteration's
    # stagnation): with this operator's conditioning (~1e7) a 1e-13 residual
    # leaves ~1e-6 in the gradient
    _, _, sv = G.gpu_setup(S, prob, tol=1e-15, max_iter=1000)
    bt = torch.as_tensor(b, device="cuda")
    xtt = torch.as_tensor(xt, device="cuda")
    x = torch.zeros_like(bt)
    sv.solve(bt, x, allow_not_converged=True)
    lam = torch.zeros_like(bt)
    sv.adjoint_solve(x - xtt, lam, allow_not_converged=True)
    dg = torch.zeros_like(bt)
    sv.diffusion_exp_gradient(torch.as_tensor(g.reshape(-1), device="cuda"), lam, x, dg)

    def solve_at(gg):
        _, _, s2 = G.gpu_setup(S, P.diffusion_from_g(gg, b), tol=1e-15, max_iter=1000)
        xx = torch.zeros_like(bt)
        s2.solve(bt, xx, allow_not_converged=True)
        return xx

    # central difference of L = 0.5 ||x - x_t||^2 summed over 2M cells: the
    # difference L+ - L- is formed as 0.5 sum (x+ - x-)(x+ + x- - 2 x_t), not
    # as a difference of two ~1e5-sized sums (whose rounding, ~1e-10, would
    # be ~5e-6 of the quotient).  What remains is the part of the two probe
    # solves' errors that does not cancel in x+ - x-: at this size it is an
    # absolute ~5e-7 in the quotient whatever the cell's derivative (the
    # quotients for h = 1e-4 and h = 5e-5 straddle the gradient ~1e-6 apart,
    # not an h^2 trend).  So the bound is norm-wise, as for the operators:
    # 2e-6 of the largest probed derivative (measured 6.8e-7; the small-size test holds 1e-6
    # per cell at h = 1e-5).
    h = 1e-4
    cells = prob.extra["fd_cells"]
    got = dg.cpu().numpy()[cells]
    scale = np.abs(got).max()
    worst = 0.0
    for c, gc in zip(cells, got):
        gp, gm = g.copy().reshape(-1), g.copy().reshape(-1)
        gp[c] += h
        gm[c] -= h
        xp, xm = solve_at(gp.reshape(g.shape)), solve_at(gm.reshape(g.shape))
        fd = 0.5 * float(((xp - xm) * (xp + xm - 2 * xtt)).sum()) / (2 * h)
        worst = max(worst, abs(fd - gc) / scale)
        assert abs(fd - gc) <= 2e-6 * scale, (c, fd, gc)
    print(f"128^3 diffusion: dL/dg vs central differences on {len(cells)} cells, "
          f"worst |fd - g| / max|g| = {worst:.2e}")


def _golden():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "var27_256_oracle.json")
    with open(path) as f:
        return json.load(f)


def test_var27_full_size_levels_and_solution_vs_oracle(S):
    """256^3 27-point, against the oracle's own full-size run (stored
    samples, tests/golden/var27_256_oracle.json, written by
    tests/golden/make_var27_256.py from oracle/ only): levels 0-4 of the
    hierarchy entry by entry at the sampled cells (every stencil entry, the
    smoother diagonal, P's weights; 1e-12 of the level's largest entry), the
    coarsening directions and level count, the FP64 PCG iteration count at
    1e-8 (within one) and its solution at the sampled cells (error stated:
    with coefficients spanning 1e8 no bound follows from the residual), and
    the FP32 cycle's."""
    gold = _golden()
    prob = P.config(2)
    _, _, sv = G.gpu_setup(S, prob, tol=1e-8, max_iter=500)
    assert sv.num_levels() == gold["num_levels"]
    for lv in gold["levels"]:
        l = lv["level"]
        n = sv.level_sizes(l)[0]
        assert n == lv["ncells"], l
        info = sv.part_info(l, 0)
        if l < gold["num_levels"] - 1:
            assert info["dstar"] == lv["dstar"], l
        cells = np.array(lv["cells"])
        ref = np.array(lv["coef"])
        got = np.zeros_like(ref)
        for ei, o in enumerate(info["offsets"]):
            code = (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1)
            got[:, code] = sv.level_copy(l, 0, 0, ei, n)[cells]
        assert np.abs(got - ref).max() <= G.OP_TOL * lv["coef_max"], l
        dinv = sv.level_copy(l, 3, n=n)[cells]
        assert G.rel(dinv, np.array(lv["dinv"])) <= G.OP_TOL, l
        if "PW" in lv:
            shp = tuple(lv["shape_zyx"])
            gW, gE = G.gpu_p(sv, l, 0, info, shp)
            assert np.abs(gW.reshape(-1)[cells] - np.array(lv["PW"])).max() <= G.OP_TOL, l
            assert np.abs(gE.reshape(-1)[cells] - np.array(lv["PE"])).max() <= G.OP_TOL, l
    bt = torch.as_tensor(prob.b[0], device="cuda")
    xc = np.array(gold["pcg"]["cells"])
    xo = np.array(gold["pcg"]["x"])
    for prec in (0, 1):
        _, _, s2 = G.gpu_setup(S, prob, precision=prec, flexible=prec, tol=1e-8, max_iter=500)
        x = torch.zeros_like(bt)
        st = s2.solve(bt, x)
        assert st.converged and st.true_rel_res <= 1.05e-8, prec
        assert abs(st.iterations - gold["pcg"]["iterations"]) <= 1, (prec, st.iterations)
        err = G.rel(x.cpu().numpy()[xc], xo)
        print(f"256^3 27-point, {'FP32 cycle' if prec else 'FP64'}: {st.iterations} iterations "
              f"(oracle {gold['pcg']['iterations']}), sampled solution error vs oracle {err:.2e}")
        assert err <= 1e-2


def test_batched_full_size_instances_vs_oracle(S):
    """The 64-problem batch at full size (its bench launch configuration):
    the eight smallest problems, every right-hand side, against the oracle's
    PCG on each problem alone: iteration counts at 1e-8 within one (both
    cycle precisions), solutions at 1e-13 (FP64 cycle, 1e-10) and 1e-12 (FP32
    cycle, 1e-9)."""
    probs = P.config(3)
    sel = sorted(range(len(probs)), key=lambda i: (probs[i].n, i))[:8]
    mats = [S.matrix_from_problem(p) for p in probs]
    nrhs = probs[0].b.shape[0]
    ref = {}
    for k in sel:
        h = O.setup(probs[k])
        for j in range(nrhs):
            ref[k, j] = (O.pcg(h, probs[k].b[j], tol=1e-8).iterations,
                         O.pcg(h, probs[k].b[j], tol=1e-13, max_iter=500).x)
    for prec, tol, stol in ((0, 1e-13, G.SOL_TOL), (1, 1e-12, 1e-9)):
        for t, check in ((1e-8, "iterations"), (tol, "solution")):
            B = S.Batch([A for _, A in mats], precision=prec, flexible=prec, tol=t, max_iter=500)
            off = B.offsets()
            bh = np.zeros((nrhs, off[-1]))
            for k, p in enumerate(probs):
                bh[:, off[k]:off[k + 1]] = p.b
            bb = torch.as_tensor(bh, device="cuda")
            xx = torch.zeros_like(bb)
            B.setup()
            st = B.solve(bb, xx, nrhs)
            xh = xx.cpu().numpy()
            for k in sel:
                for j in range(nrhs):
                    if check == "iterations":
                        assert abs(st[j][k].iterations - ref[k, j][0]) <= 1, (prec, k, j)
                    else:
                        assert G.rel(xh[j, off[k]:off[k + 1]], ref[k, j][1]) <= stol, (prec, k, j)
            del B
