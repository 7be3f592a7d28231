"""Batching form: many independent problems and right-hand sides together.

Each (problem, right-hand side) instance of a batch solve is compared with
the oracle's PCG on that problem alone: solutions run to 1e-13 agree to 1e-10
relative, iteration counts at the 1e-8 stop agree within one.  The union
hierarchy carries a problem whose parts reach one cell early through identity
levels down to an exact coarsest solve, so its preconditioner is the
problem's own up to rounding.
"""
import numpy as np
import pytest

import problems as P
from oracle import ssamg as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S(ssamg_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ssamg_lib


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def make_batch(S, probs, **kw):
    mats = [S.matrix_from_problem(p) for p in probs]
    B = S.Batch([A for _, A in mats], **kw)
    B.setup()
    return mats, B


def stack_rhs(probs, off, nrhs):
    N = off[-1]
    b = np.zeros((nrhs, N))
    for k, p in enumerate(probs):
        for j in range(nrhs):
            b[j, off[k]:off[k + 1]] = p.b[j]
    return b


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_oracle_per_instance(S, prec):
    probs = P.config(3, small=True)
    nrhs = probs[0].b.shape[0]
    mats, B = make_batch(S, probs, precision=prec, flexible=prec, tol=1e-13, max_iter=500)
    off = B.offsets()
    assert off[-1] == sum(p.n for p in probs) == B.num_cells()
    b = torch.as_tensor(stack_rhs(probs, off, nrhs), device="cuda").contiguous()
    x = torch.zeros_like(b)
    st = B.solve(b, x, nrhs)
    xs = x.cpu().numpy()
    hs = [O.setup(p) for p in probs]
    for k, p in enumerate(probs):
        for j in range(nrhs):
            ref = O.pcg(hs[k], p.b[j], tol=1e-13, max_iter=500)
            assert st[j][k].converged and st[j][k].true_rel_res <= 1e-12
            assert rel(xs[j, off[k]:off[k + 1]], ref.x) <= 1e-10, (k, j)

    _, B8 = make_batch(S, probs, precision=prec, flexible=prec)
    x8 = torch.zeros_like(b)
    st8 = B8.solve(b, x8, nrhs)
    for k, p in enumerate(probs):
        for j in range(nrhs):
            ref = O.pcg(hs[k], p.b[j], tol=1e-8)
            assert abs(st8[j][k].iterations - ref.iterations) <= 1, (k, j)
            assert st8[j][k].rel_res <= 1e-8


def test_batch_of_one_is_the_solver(S):
    prob = P.multipart_aniso(m=9, layout=(2, 1, 2), seed=7)
    _, A = S.matrix_from_problem(prob)
    B = S.Batch([A], precision=1, flexible=1)
    B.setup()
    sv = S.Solver(precision=1, flexible=1)
    sv.setup(A)
    b = torch.as_tensor(prob.b[0], device="cuda")
    xb = torch.zeros_like(b)
    xs = torch.zeros_like(b)
    stb = B.solve(b, xb)
    sts = sv.solve(b, xs)
    assert stb[0][0].iterations == sts.iterations
    assert torch.equal(xb, xs)


def test_batch_zero_rhs_instance_stays_zero(S):
    probs = P.batched(nprob=4, nrhs=1, seed=11, pmax=3, emin=3, emax=9)
    mats, B = make_batch(S, probs)
    off = B.offsets()
    bh = stack_rhs(probs, off, 1)
    bh[0, off[2]:off[3]] = 0.0
    b = torch.as_tensor(bh, device="cuda").contiguous()
    x = torch.zeros_like(b)
    st = B.solve(b, x)
    assert st[0][2].iterations == 0 and float(x[0, off[2]:off[3]].abs().max()) == 0.0
    for k in (0, 1, 3):
        assert st[0][k].converged and st[0][k].iterations > 0


def test_batch_rejects_mixed_stencils(S):
    a = P.laplace7(4)
    c = P.var27(n=5, block=5, seed=2)
    _, A1 = S.matrix_from_problem(a)
    _, A2 = S.matrix_from_problem(c)
    with pytest.raises(S.SsamgError):
        S.Batch([A1, A2])


def test_batch_one_graph_matches_host_loop(S):
    """All right-hand sides in one graph launch (cached per vector pair, and
    rebuilt for new vectors) give the host-driven rounds' results bitwise."""
    probs = P.batched(nprob=5, nrhs=3, seed=13, pmax=3, emin=4, emax=11)
    res = []
    for graph in (1, 0):
        _, B = make_batch(S, probs, precision=1, flexible=1, use_graph=graph)
        off = B.offsets()
        b = torch.as_tensor(stack_rhs(probs, off, 3), device="cuda").contiguous()
        x = torch.zeros_like(b)
        st = B.solve(b, x, 3)
        x2 = torch.zeros_like(b)
        st2 = B.solve(b, x2, 3)         # new output vector: the graph is rebuilt
        x.zero_()
        st3 = B.solve(b, x, 3)          # same vectors again: the cached graph
        assert torch.equal(x, x2)
        its = [[s.iterations for s in row] for row in st]
        assert its == [[s.iterations for s in row] for row in st2]
        assert its == [[s.iterations for s in row] for row in st3]
        res.append((its, x.cpu().numpy()))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


@pytest.mark.parametrize("prec,use_tail,bricks,kind", [
    (1, 3, 1, "7pt"), (0, 3, 1, "7pt"), (1, 0, 1, "7pt"), (1, 3, 0, "7pt"),
    (0, 0, 0, "7pt"), (1, 3, 1, "27pt"), (0, 0, 1, "27pt"), (1, 2, 1, "7pt")])
def test_rhs_together_matches_one_after_another(S, prec, use_tail, bricks, kind):
    """Right-hand sides solved in one PCG loop (the residual and relaxation
    of cell-tile levels taking all of them per launch) give each right-hand
    side's one-after-another results bitwise: solutions, iteration counts,
    residuals and the last right-hand side's residual history."""
    if kind == "7pt":
        probs = P.batched(nprob=4, nrhs=3, seed=17, pmax=3, emin=4, emax=12)
    else:
        probs = [P.var27(n=n, block=3, seed=20 + n, nrhs=3) for n in (7, 9, 6)]
    res = []
    for together in (1, 0):
        _, B = make_batch(S, probs, precision=prec, flexible=prec, use_tail=use_tail,
                          tail_cells=256, use_bricks=bricks, rhs_together=together)
        off = B.offsets()
        b = torch.as_tensor(stack_rhs(probs, off, 3), device="cuda").contiguous()
        x = torch.zeros_like(b)
        st = B.solve(b, x, 3)
        its = [[(s.iterations, s.rel_res, s.true_rel_res) for s in row] for row in st]
        hist = [B.solver().residual_history(k) for k in range(len(probs))]
        # fewer right-hand sides next (the slices of the first solve are reused)
        b2 = b[:2].contiguous()
        x2 = torch.zeros_like(b2)
        st2 = B.solve(b2, x2, 2)
        its.append([[s.iterations for s in row] for row in st2])
        res.append((its, np.concatenate([x.cpu().numpy(), x2.cpu().numpy()]), hist,
                    st[0][0].solve_kernel_launches))
    # together, one loop enqueues every right-hand side's steps (a fused
    # single-CTA tail, where the batch has one, takes them one after another)
    if use_tail != 2:
        assert res[0][3] > res[1][3]
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])
    for h0, h1 in zip(res[0][2], res[1][2]):
        assert np.array_equal(h0, h1)
