"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Operators (W, d*, omega, P, A_c = P^T S P + P^T U P, smoother diagonals) are
compared level by level with max|gpu - oracle| <= 1e-12 max|oracle| (the
per-level norm-wise form; FP64 on both sides, only the summation order
differs).  Solutions of runs taken to a 1e-13 residual agree to 1e-10
relative; iteration counts at the 1e-8 stop agree within one.  The FP32 cycle
(precision 1) is compared with the FP64 cycle to 5e-5 relative (single
precision roundoff amplified by the level operators' conditioning) and must
still reach the same FP64 solution.
"""
import numpy as np
import pytest

import problems as P
from oracle import ssamg as O

import test_oracle as T

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OP_TOL = 1e-12
SOL_TOL = 1e-10


@pytest.fixture(scope="module")
def S(ssamg_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ssamg_lib


def cases():
    out = list(T.SMALL)
    out += [
        P.laplace7(20),                                    # several tiles + ragged tail
        P.multipart_aniso(m=11, layout=(2, 2, 2), seed=1),
        T.chain([7, 13, 10], [[.3, 1, .2], [1, .1, .1], [.05, .5, 1]]),
        P.var27(n=13, block=3, seed=2),
        P.diffusion_exp(n=12, seed=4, nfd=2),
        T.shifted(P.multipart_aniso(m=6, layout=(1, 2, 2), seed=5), [(-5, 3, 1), (2, 2, -3), (0, 0, 0), (7, -1, 2)]),
        T.chain([1, 4], [[1, 1, 1], [1, .5, .2]]),         # a one-cell part
        T.poisson2d(9, 4),
        P.three_point(9),                                  # rotated index maps (test case 3)
        P.samr(12),                                        # ghost unknowns, inner rows (test case 4)
        P.multibox(9),                                     # a part of two boxes (Section 2)
    ]
    for k in range(5):
        c = P.config(k, small=True)
        out += c if isinstance(c, list) else [c]
    return out


CASES = cases()
CIDS = [f"{i}-{p.name}" for i, p in enumerate(CASES)]


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    s = max(np.abs(b).max(initial=0.0), 1e-300)
    return np.abs(a - b).max(initial=0.0) / s


def gpu_setup(S, prob, **kw):
    grid, A = S.matrix_from_problem(prob)
    solver = S.Solver(**kw)
    solver.setup(A)
    return grid, A, solver


def gpu_level(S, solver, l, nparts):
    """One level of the GPU hierarchy in the oracle's form."""
    n, nr, nnz = solver.level_sizes(l)
    lev = {"n": n, "parts": []}
    for p in range(nparts):
        info = solver.part_info(l, p)
        lo, hi = np.array(info["lo"]), np.array(info["hi"])
        e = hi - lo + 1
        shp = (int(e[2]), int(e[1]), int(e[0]))
        ncell = int(np.prod(shp))
        st = {}
        for ei, o in enumerate(info["offsets"]):
            st[tuple(o)] = solver.level_copy(l, 0, p, ei, ncell).reshape(shp)
        info["S"] = st
        info["shape"] = shp
        lev["parts"].append(info)
    lev["dinv"] = solver.level_copy(l, 3, n=n)
    if nr:
        ptr = solver.level_copy(l, 4, n=nr + 1, dtype=np.int32)
        rows = solver.level_copy(l, 5, n=nr, dtype=np.int32)
        cols = solver.level_copy(l, 6, n=nnz, dtype=np.int32)
        vals = solver.level_copy(l, 7, n=nnz)
        bits = solver.level_copy(l, 8, n=nnz, dtype=np.uint8)
        r = np.repeat(rows, np.diff(ptr))
        lev["U"] = {(int(a), int(b)): (float(v), int(t)) for a, b, v, t in zip(r, cols, vals, bits)}
    else:
        lev["U"] = {}
    return lev


def gpu_p(solver, l, p, info, fine_shape):
    """P weights of a coarsened part scattered back onto the fine grid."""
    d = info["dstar"]
    par = info["lo"][d] & 1
    nf = list(fine_shape[::-1])  # x, y, z
    nf[d] = (nf[d] + par) >> 1
    cnt = int(np.prod(nf))
    out = []
    for what in (1, 2):
        w = solver.level_copy(l, what, p, 0, cnt).reshape(nf[2], nf[1], nf[0])
        full = np.zeros(fine_shape)
        ax = 2 - d
        idx = 2 * np.arange(nf[d]) + 1 - par
        sl = [slice(None)] * 3
        sl[ax] = idx
        full[tuple(sl)] = w
        out.append(full)
    return out


def compare_hierarchy(S, prob, solver, h):
    assert solver.num_levels() == len(h.levels)
    c, W = solver.spacings(prob.nparts)
    cref = O.coupling_sums(h.levels[0])
    assert rel(c, cref) <= 1e-13
    fin = np.isfinite(h.W0)
    assert np.array_equal(np.isfinite(W), fin)
    assert rel(W[fin], h.W0[fin]) <= 1e-13
    for l, lev in enumerate(h.levels):
        g = gpu_level(S, solver, l, prob.nparts)
        assert g["n"] == lev.n
        for p in range(lev.nparts):
            gi = g["parts"][p]
            assert tuple(gi["lo"]) == tuple(lev.lo[p]) and tuple(gi["hi"]) == tuple(lev.hi[p]), (l, p)
            assert gi["dstar"] == lev.dstar[p], (l, p)
            assert abs(gi["omega"] - lev.omega[p]) <= 1e-14, (l, p)
            keys = set(gi["S"]) | set(lev.S[p])
            scale = max(np.abs(a).max() for a in lev.S[p].values())
            for o in keys:
                a = gi["S"].get(o, np.zeros(lev.shape(p)))
                b = lev.S[p].get(o, np.zeros(lev.shape(p)))
                if not isinstance(b, np.ndarray):
                    b = np.full(lev.shape(p), float(b))
                b = np.where(O._inside_mask(lev.shape(p), o), b, 0.0)
                a = np.where(O._inside_mask(lev.shape(p), o), a, 0.0)
                assert np.abs(a - b).max() <= OP_TOL * scale, (l, p, o)
            if lev.dstar[p] >= 0:
                PW, PE = gpu_p(solver, l, p, gi, lev.shape(p))
                assert np.abs(PW - lev.PW[p]).max() <= OP_TOL, (l, p)
                assert np.abs(PE - lev.PE[p]).max() <= OP_TOL, (l, p)
        assert rel(g["dinv"], lev.Dinv) <= OP_TOL, l
        ref_u = {(int(a), int(b)): (float(v), int(t)) for a, b, v, t in
                 zip(lev.u_row, lev.u_col, lev.u_val, lev.u_bits)}
        if ref_u or g["U"]:
            scale = max(abs(v) for v, _ in ref_u.values())
            for k in set(ref_u) | set(g["U"]):
                va, ta = g["U"].get(k, (0.0, 0))
                vb, tb = ref_u.get(k, (0.0, 0))
                assert abs(va - vb) <= OP_TOL * scale, (l, k)
            assert set(ref_u) == set(g["U"]), l
            assert all(g["U"][k][1] == ref_u[k][1] for k in ref_u), l


@pytest.mark.parametrize("prob", CASES, ids=CIDS)
def test_hierarchy_matches_oracle(S, prob):
    h = O.setup(prob)
    grid, A, solver = gpu_setup(S, prob)
    compare_hierarchy(S, prob, solver, h)


@pytest.mark.parametrize("prob", CASES, ids=CIDS)
def test_hierarchy_l1_fp32_matches_oracle(S, prob):
    h = O.setup(prob, O.Params(relax=1))
    grid, A, solver = gpu_setup(S, prob, relax=1, precision=1)
    compare_hierarchy(S, prob, solver, h)


@pytest.mark.parametrize("prob", CASES, ids=CIDS)
def test_vcycle_and_matvec_match_oracle(S, prob):
    h = O.setup(prob)
    r = P.SplitMix64(17).uniform_pm1(prob.n)
    rt = torch.as_tensor(r, device="cuda")
    zr = O.vcycle(h, r)
    # one launch per level and step (default), the cooperative-grid tail, the
    # single-CTA tail and the assembled coarse levels in one cluster
    for tail in (0, 1, 2, 3):
        grid, A, solver = gpu_setup(S, prob, use_tail=tail)
        z = torch.zeros_like(rt)
        solver.precondition(rt, z)
        assert rel(z.cpu().numpy(), zr) <= OP_TOL, tail
    for l, lev in enumerate(h.levels):
        x = P.SplitMix64(l).uniform_pm1(lev.n)
        y = torch.zeros(lev.n, dtype=torch.float64, device="cuda")
        solver.level_matvec(l, torch.as_tensor(x, device="cuda"), y)
        assert rel(y.cpu().numpy(), O.matvec(lev, x)) <= OP_TOL, l
    # FP32 cycle against the FP64 cycle
    for tail in (0, 1, 2, 3):
        _, _, s32 = gpu_setup(S, prob, precision=1, use_tail=tail)
        z32 = torch.zeros_like(rt)
        s32.precondition(rt, z32)
        assert rel(z32.cpu().numpy(), zr) <= 5e-5, tail


@pytest.mark.parametrize("prob", CASES, ids=CIDS)
def test_pcg_matches_oracle(S, prob):
    h = O.setup(prob)
    b = prob.b[0]
    bt = torch.as_tensor(b, device="cuda")
    tight = O.pcg(h, b, tol=1e-13, max_iter=500)
    at8 = O.pcg(h, b, tol=1e-8)
    for graph, tail in ((1, 1), (0, 0), (1, 2), (1, 3), (0, 3)):
        grid, A, solver = gpu_setup(S, prob, tol=1e-13, max_iter=500, use_graph=graph, use_tail=tail)
        x = torch.zeros_like(bt)
        st = solver.solve(bt, x)
        assert st.converged
        assert rel(x.cpu().numpy(), tight.x) <= SOL_TOL
        assert st.true_rel_res <= 1e-12
        _, _, s8 = gpu_setup(S, prob, use_graph=graph, use_tail=tail)
        x8 = torch.zeros_like(bt)
        st8 = s8.solve(bt, x8)
        assert abs(st8.iterations - at8.iterations) <= 1, (st8.iterations, at8.iterations)
        assert st8.rel_res <= 1e-8


@pytest.mark.parametrize("prob", CASES, ids=CIDS)
def test_mixed_precision_reaches_fp64_solution(S, prob):
    h = O.setup(prob)
    b = prob.b[0]
    tight = O.pcg(h, b, tol=1e-12, max_iter=500)
    grid, A, solver = gpu_setup(S, prob, precision=1, flexible=1, tol=1e-12, max_iter=500)
    bt = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bt)
    st = solver.solve(bt, x)
    assert st.converged and st.true_rel_res <= 1e-11
    assert rel(x.cpu().numpy(), tight.x) <= 1e-9


def test_solve_host_and_multiple_rhs(S):
    prob = P.multipart_aniso(m=7, layout=(2, 1, 2), seed=3, nrhs=3)
    h = O.setup(prob)
    grid, A, solver = gpu_setup(S, prob, tol=1e-12)
    b = np.ascontiguousarray(prob.b.reshape(-1))
    x = np.zeros_like(b)
    solver.solve_host(b, x, nrhs=3)
    bt = torch.as_tensor(b, device="cuda")
    xt = torch.zeros_like(bt)
    solver.solve(bt, xt, nrhs=3)
    for k in range(3):
        ref = O.pcg(h, prob.b[k], tol=1e-12).x
        assert rel(x[k * prob.n:(k + 1) * prob.n], ref) <= 1e-9
        assert rel(xt.cpu().numpy()[k * prob.n:(k + 1) * prob.n], ref) <= 1e-9


def test_nonzero_initial_guess_and_resetup(S):
    prob = P.multipart_aniso(m=6, layout=(2, 2, 1), seed=2)
    h = O.setup(prob)
    grid, A, solver = gpu_setup(S, prob, tol=1e-12)
    bt = torch.as_tensor(prob.b[0], device="cuda")
    ref = O.pcg(h, prob.b[0], tol=1e-12).x
    x0 = torch.as_tensor(ref + 1e-3 * P.SplitMix64(1).uniform_pm1(prob.n), device="cuda")
    st = solver.solve(bt, x0, zero_guess=False)
    assert rel(x0.cpu().numpy(), ref) <= 1e-9
    for _ in range(2):       # setting up again reuses the same device memory
        solver.setup(A)
        x = torch.zeros_like(bt)
        solver.solve(bt, x)
        assert rel(x.cpu().numpy(), ref) <= 1e-9


def test_options_coarse_relax_and_level_caps(S):
    prob = P.multipart_aniso(m=5, layout=(2, 1, 1), seed=4)
    for kw, okw in (({"coarse_direct": 0}, {"coarse_direct": 0}),
                    ({"max_levels": 3}, {"max_levels": 3}),
                    ({"s_max": 40}, {"s_max": 40}),
                    ({"max_levels": 1}, {"max_levels": 1}),
                    ({"relax_factor": 0.7}, {"relax_factor": 0.7}),
                    ({"relax": 1, "relax_factor": 1.2}, {"relax": 1, "relax_factor": 1.2})):
        h = O.setup(prob, O.Params(**okw))
        grid, A, solver = gpu_setup(S, prob, tol=1e-12, max_iter=400, **kw)
        compare_hierarchy(S, prob, solver, h)
        r = P.SplitMix64(3).uniform_pm1(prob.n)
        z = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        solver.precondition(torch.as_tensor(r, device="cuda"), z)
        assert rel(z.cpu().numpy(), O.vcycle(h, r)) <= OP_TOL, kw


def test_breakdown_is_reported(S):
    """An indefinite operator ends in a status, not a hang or a fault."""
    prob = P.laplace7(6)
    prob.coef[0][0] = -6.0
    grid, A = S.matrix_from_problem(prob)
    solver = S.Solver()
    with pytest.raises(S.SsamgError) as e:
        solver.setup(A)
        bt = torch.as_tensor(prob.b[0], device="cuda")
        solver.solve(bt, torch.zeros_like(bt))
    assert e.value.code in (S.ERR_BREAKDOWN,)


def test_nan_rhs_is_reported(S):
    prob = P.laplace7(6)
    grid, A, solver = gpu_setup(S, prob)
    b = prob.b[0].copy()
    b[5] = np.nan
    bt = torch.as_tensor(b, device="cuda")
    with pytest.raises(S.SsamgError) as e:
        solver.solve(bt, torch.zeros_like(bt))
    assert e.value.code == S.ERR_BREAKDOWN


@pytest.mark.parametrize("prob", [P.multipart_aniso(m=6, layout=(2, 1, 2), seed=6),
                                  P.var27(n=7, block=3, seed=2)], ids=["aniso", "var27"])
def test_coef_gradient_matches_oracle(S, prob):
    """dL/da per stencil entry, in the user's entry order (a 27-point
    stencil is held internally in offset-code order)."""
    h = O.setup(prob)
    grid, A, solver = gpu_setup(S, prob)
    lam = P.SplitMix64(1).uniform_pm1(prob.n)
    x = P.SplitMix64(2).uniform_pm1(prob.n)
    k = len(prob.offsets)
    d = torch.zeros(k * prob.n, dtype=torch.float64, device="cuda")
    solver.coef_gradient(torch.as_tensor(lam, device="cuda"), torch.as_tensor(x, device="cuda"), d)
    d = d.cpu().numpy().reshape(k, prob.n)
    ref = O.coef_gradient(h.levels[0], lam, x)
    offs = h.levels[0].offsets()
    for e, o in enumerate(prob.offsets):
        o = tuple(int(v) for v in o)
        for p in range(prob.nparts):
            assert rel(d[e, offs[p]:offs[p + 1]], ref[p][o].reshape(-1)) <= 1e-15


def test_diffusion_gradient_matches_oracle_and_fd(S):
    prob = P.diffusion_exp(n=10, seed=4, nfd=6)
    g, xt, b = prob.extra["g"], prob.extra["x_t"], prob.b[0]
    h = O.setup(prob)
    grid, A, solver = gpu_setup(S, prob, tol=1e-13, max_iter=400)
    bt = torch.as_tensor(b, device="cuda")
    x = torch.zeros_like(bt)
    solver.solve(bt, x)
    lam = torch.zeros_like(bt)
    solver.adjoint_solve(x - torch.as_tensor(xt, device="cuda"), lam)
    dg = torch.zeros_like(bt)
    solver.diffusion_exp_gradient(torch.as_tensor(g.reshape(-1), device="cuda"), lam, x, dg)
    xo = O.pcg(h, b, tol=1e-13).x
    lo = O.pcg(h, xo - xt, tol=1e-13).x
    ref = O.diffusion_exp_gradient(g, lo, xo).reshape(-1)
    assert rel(dg.cpu().numpy(), ref) <= 1e-9

    def loss(gg):
        pr = P.diffusion_from_g(gg, b)
        _, AA, sv = gpu_setup(S, pr, tol=1e-14, max_iter=400)
        xx = torch.zeros_like(bt)
        sv.solve(bt, xx, allow_not_converged=True)
        return 0.5 * float(((xx.cpu().numpy() - xt) ** 2).sum())

    for c in prob.extra["fd_cells"][:4]:
        hstep = 1e-5
        gp = g.copy().reshape(-1)
        gm = g.copy().reshape(-1)
        gp[c] += hstep
        gm[c] -= hstep
        fd = (loss(gp.reshape(g.shape)) - loss(gm.reshape(g.shape))) / (2 * hstep)
        got = dg.cpu().numpy()[c]
        assert abs(fd - got) <= 1e-6 * max(abs(fd), 1e-6), (c, fd, got)


@pytest.mark.parametrize("prec", [0, 1])
def test_programmatic_launch_matches_plain_launches(S, prec):
    """Programmatic dependent launch only changes when kernels are scheduled:
    every kernel still waits for its predecessor before touching the solve's
    vectors, so the result is bitwise that of plain launches (graph and host
    loop alike)."""
    prob = P.multipart_aniso(m=24, layout=(2, 2, 2), seed=1)
    b = torch.as_tensor(prob.b[0], device="cuda")
    runs = []
    for pdl in (0, 1):
        for graph in (0, 1):
            _, _, sv = gpu_setup(S, prob, precision=prec, flexible=prec, use_pdl=pdl,
                                 use_graph=graph)
            x = torch.zeros_like(b)
            st = sv.solve(b, x)
            assert st.converged
            z = torch.zeros_like(b)
            sv.precondition(b, z)
            runs.append((st.iterations, x.cpu().numpy(), z.cpu().numpy()))
    for it, x, z in runs[1:]:
        assert it == runs[0][0]
        assert np.array_equal(x, runs[0][1])
        assert np.array_equal(z, runs[0][2])


@pytest.mark.parametrize("prob", [CASES[i] for i in (0, 13, 17, 18, 20)],
                         ids=[CIDS[i] for i in (0, 13, 17, 18, 20)])
@pytest.mark.parametrize("prec", [0, 1])
def test_brick_applies_match_cell_tiles(S, prob, prec):
    """Checked 7-point levels run their operator applies over z-marching
    bricks; a cell's A x is summed in the same order as on the cell tiles, so
    the V-cycle is bitwise the same, and the PCG (whose dot partials group
    cells differently) converges in the same number of iterations."""
    r = torch.as_tensor(P.SplitMix64(41).uniform_pm1(prob.n), device="cuda")
    b = torch.as_tensor(prob.b[0], device="cuda")
    zs, runs = [], []
    for bricks in (0, 1):
        _, _, sv = gpu_setup(S, prob, precision=prec, flexible=prec, use_bricks=bricks,
                             tol=1e-12, max_iter=500)
        z = torch.zeros_like(r)
        sv.precondition(r, z)
        zs.append(z.cpu().numpy())
        x = torch.zeros_like(b)
        st = sv.solve(b, x)
        runs.append((st.iterations, x.cpu().numpy()))
    assert np.array_equal(zs[0], zs[1])
    assert abs(runs[0][0] - runs[1][0]) <= 1
    assert rel(runs[1][1], runs[0][1]) <= 1e-9


@pytest.mark.parametrize("prob", [CASES[i] for i in (0, 13, 20)] + [P.laplace7(16)],
                         ids=[CIDS[i] for i in (0, 13, 20)] + ["laplace7 16^3"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("mode", [1, 2])
def test_skip_option_matches_oracle(S, prob, prec, mode):
    """Section 3.4 "skip" (mode 1: rounds of distinct directions; mode 2: the
    printed test alone): the hierarchy (skipped parts' smoothers zero), one
    V-cycle and the PCG iteration count against the oracle with skip on."""
    h = O.setup(prob, O.Params(skip=mode))
    _, _, sv = gpu_setup(S, prob, skip=mode, precision=prec, flexible=prec)
    if prec == 0:
        compare_hierarchy(S, prob, sv, h)
    r = P.SplitMix64(43).uniform_pm1(prob.n)
    z = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    sv.precondition(torch.as_tensor(r, device="cuda"), z)
    assert rel(z.cpu().numpy(), O.vcycle(h, r)) <= (OP_TOL if prec == 0 else 5e-5)
    ref = O.pcg(h, prob.b[0], tol=1e-8)
    x = torch.zeros_like(z)
    st = sv.solve(torch.as_tensor(prob.b[0], device="cuda"), x)
    assert abs(st.iterations - ref.iterations) <= 1, (st.iterations, ref.iterations)


@pytest.mark.parametrize("prob", [CASES[i] for i in (0, 2, 5, 13, 14, 15, 18, 19)],
                         ids=[CIDS[i] for i in (0, 2, 5, 13, 14, 15, 18, 19)])
@pytest.mark.parametrize("cells", [64, 512, 4096])
def test_cluster_tail_matches_oracle(S, prob, cells):
    """The coarse-level transition (use_tail = 3, Section 3.5's hybrid idea):
    the levels from the first of at most `cells` cells down are assembled
    (A = S + U, P, P^T, smoother diagonal, coarsest inverse) and run in one
    thread-block cluster.  The V-cycle is the same operation, so it matches
    the oracle's at 1e-12 (FP64) and 5e-5 (FP32 cycle); with the relaxation
    sweep on the coarsest level too; PCG iterations at 1e-8 within one; and
    the tail really runs (its first level is the first of at most `cells`
    cells below level 0)."""
    h = O.setup(prob)
    r = P.SplitMix64(23).uniform_pm1(prob.n)
    rt = torch.as_tensor(r, device="cuda")
    zr = O.vcycle(h, r)
    sizes = [lev.n for lev in h.levels]
    want = next((l for l in range(1, len(sizes)) if sizes[l] <= cells), len(sizes) - 1)
    for prec, tol in ((0, OP_TOL), (1, 5e-5)):
        _, _, sv = gpu_setup(S, prob, precision=prec, flexible=prec, use_tail=3, tail_cells=cells)
        first, nlev = sv.tail_levels()
        if want < len(sizes) - 1:
            assert first == want and nlev == len(sizes) - want, (first, nlev, sizes)
        else:
            assert nlev == 0
        z = torch.zeros_like(rt)
        sv.precondition(rt, z)
        assert rel(z.cpu().numpy(), zr) <= tol, prec
        z2 = torch.zeros_like(rt)
        sv.precondition(rt, z2)
        assert torch.equal(z, z2)   # bit for bit from run to run
    h0 = O.setup(prob, O.Params(coarse_direct=0))
    _, _, sv = gpu_setup(S, prob, use_tail=3, tail_cells=cells, coarse_direct=0)
    z = torch.zeros_like(rt)
    sv.precondition(rt, z)
    assert rel(z.cpu().numpy(), O.vcycle(h0, r)) <= OP_TOL
    ref = O.pcg(h, prob.b[0], tol=1e-8)
    _, _, sv = gpu_setup(S, prob, precision=1, flexible=1, use_tail=3, tail_cells=cells)
    x = torch.zeros_like(rt)
    st = sv.solve(torch.as_tensor(prob.b[0], device="cuda"), x)
    assert st.converged and abs(st.iterations - ref.iterations) <= 1


def _split_couplings(prob, seed=11):
    """The same matrix with every coupling given twice (value halves, exact)
    and the coupling list shuffled."""
    import dataclasses
    m = prob.nnz_u
    rng = np.random.default_rng(seed)
    perm = rng.permutation(2 * m)
    rep = lambda a: np.concatenate([a, a])[perm]
    return dataclasses.replace(prob, u_part=rep(prob.u_part), u_idx=rep(prob.u_idx),
                               u_dir=rep(prob.u_dir), u_nbor_part=rep(prob.u_nbor_part),
                               u_nbor_idx=rep(prob.u_nbor_idx), u_val=rep(prob.u_val * 0.5))


@pytest.mark.parametrize("prob", [P.multipart_aniso(m=7, layout=(2, 2, 1), seed=3), P.samr(8),
                                  P.three_point(5)], ids=["aniso4", "samr", "tc3"])
def test_duplicate_and_unordered_couplings_assemble_the_same_rows(S, prob):
    """Matrix assembly sorts couplings by row and column and sums duplicates:
    a shuffled list with every coupling split in two exact halves gives the
    same level-0 coupling rows, bit for bit, and the same hierarchy."""
    _, _, sv1 = gpu_setup(S, prob)
    _, _, sv2 = gpu_setup(S, _split_couplings(prob))
    u1 = gpu_level(S, sv1, 0, prob.nparts)["U"]
    u2 = gpu_level(S, sv2, 0, prob.nparts)["U"]
    assert u1 == u2 and len(u1) > 0
    for l in range(1, sv1.num_levels()):
        a = gpu_level(S, sv1, l, prob.nparts)
        b = gpu_level(S, sv2, l, prob.nparts)
        assert a["U"] == b["U"]
        for pa, pb in zip(a["parts"], b["parts"]):
            for o in pa["S"]:
                assert np.array_equal(pa["S"][o], pb["S"][o])


def test_device_cache_release_after_objects(S):
    """Objects destroyed leave their device memory to the pool; releasing it
    returns the cached bytes, a second release returns nothing, and a new
    matrix and solver still work afterwards."""
    import gc
    prob = P.multipart_aniso(m=6, layout=(2, 1, 1), seed=1)
    for _ in range(2):
        _, _, sv = gpu_setup(S, prob)
        del sv
        gc.collect()
    torch.cuda.synchronize()
    first = S.lib().ssamg_release_device_cache()
    assert first > 0
    assert S.lib().ssamg_release_device_cache() == 0
    h = O.setup(prob)
    _, _, sv = gpu_setup(S, prob)
    compare_hierarchy(S, prob, sv, h)


@pytest.mark.parametrize("prob,W", [
    (P.multipart_aniso(m=11, layout=(2, 2, 2), seed=1), np.ones((8, 3))),
    (P.laplace7(13), np.array([[1.0, 1.0, 0.5]])),
    (P.three_point(7), np.array([[1.0, np.inf, 1.0], [0.5, 1.0, 1.0], [1.0, 1.0, 1.0]])),
], ids=["aniso8-isotropic-W", "cube-W", "tc3-W"])
def test_user_spacings_match_oracle(S, prob, W):
    """Representative grid spacings given by the user (Section 3.1) replace
    the computed ones in Algorithm 1 and Eq. relax1, on both sides."""
    h = O.setup(prob, O.Params(spacings=W))
    grid, A = S.matrix_from_problem(prob)
    sv = S.Solver()
    sv.set_spacings(W)
    sv.setup(A)
    compare_hierarchy(S, prob, sv, h)   # W compared with the oracle's W0: the user's
    b = torch.as_tensor(prob.b[0], device="cuda")
    x = torch.zeros_like(b)
    st = sv.solve(b, x)
    ref = O.pcg(h, prob.b[0], tol=1e-8)
    assert abs(st.iterations - ref.iterations) <= 1
    # back to the computed spacings
    sv.set_spacings(None)
    sv.setup(A)
    compare_hierarchy(S, prob, sv, O.setup(prob))


def test_user_spacings_rejected(S):
    grid, A = S.matrix_from_problem(P.laplace7(6))
    sv = S.Solver()
    with pytest.raises(S.SsamgError):
        sv.set_spacings(np.array([[1.0, float("nan"), 1.0]]))
    sv.set_spacings(np.ones((2, 3)))          # one part in the grid
    with pytest.raises(S.SsamgError):
        sv.setup(A)


@pytest.mark.parametrize("prob", [P.multipart_aniso(m=11, layout=(2, 2, 2), seed=1),
                                  P.samr(8)], ids=["aniso8", "samr"])
def test_residual_history_matches_oracle(S, prob):
    """||r_k|| / ||b|| of every iteration (FP64 cycle) against the oracle's
    PCG history: the same iteration count, each value to 1e-9 relative (the
    recursive residuals of two FP64 runs that differ in summation order)."""
    grid, A, sv = gpu_setup(S, prob, tol=1e-8)
    b = torch.as_tensor(prob.b[0], device="cuda")
    x = torch.zeros_like(b)
    st = sv.solve(b, x)
    hist = sv.residual_history()
    ref = O.pcg(O.setup(prob), prob.b[0], tol=1e-8)
    assert len(hist) == st.iterations + 1 == len(ref.history)
    assert hist[0] == pytest.approx(1.0, rel=1e-14)
    assert abs(hist[-1] - st.rel_res) <= 1e-15 * max(st.rel_res, 1e-300) * 10
    h = np.array(ref.history)
    assert np.all(np.abs(hist - h) <= 1e-9 * h + 1e-300)
    assert S.lib().ssamg_residual_history(sv.h, 1, None, 4) == S.ERR_ARG


@pytest.mark.parametrize("kind", ["27pt", "7pt"])
def test_solve_several_rhs_one_graph(S, kind):
    """ssamg_solve with several right-hand sides runs them in one graph
    launch (together where the hierarchy allows it), from zero or from given
    initial guesses: each solution bitwise that of its own solve, and within
    1e-9 of the oracle's."""
    if kind == "27pt":
        prob = P.var27(n=24, block=4, seed=31, nrhs=3)
    else:
        prob = P.multipart_aniso(m=16, layout=(2, 1, 2), seed=5, nrhs=3)
    grid, A, solver = gpu_setup(S, prob, precision=1, flexible=1, tol=1e-12)
    n = prob.n
    bt = torch.as_tensor(np.ascontiguousarray(prob.b.reshape(-1)), device="cuda")
    x0 = torch.as_tensor(P.SplitMix64(9).uniform_pm1(3 * n) * 1e-2, device="cuda")
    for zero in (True, False):
        x = torch.zeros_like(bt) if zero else x0.clone()
        st = solver.solve(bt, x, nrhs=3, zero_guess=zero)
        assert st.converged
        for k in range(3):
            xk = torch.zeros(n, dtype=torch.float64, device="cuda") if zero \
                else x0[k * n:(k + 1) * n].clone()
            sk = solver.solve(bt[k * n:(k + 1) * n].contiguous(), xk, zero_guess=zero)
            assert torch.equal(x[k * n:(k + 1) * n], xk), (zero, k)
        assert sk.iterations == st.iterations  # the last right-hand side's stats
    h = O.setup(prob)
    for k in range(3):
        ref = O.pcg(h, prob.b[k], tol=1e-12).x
        assert rel(x[k * n:(k + 1) * n].cpu().numpy(), ref) <= 1e-9
