"""Tile forms and the tile autotuner.

A tile form (cells per thread, bricks) decides only which thread computes
which cell, so every V-cycle result must be the same bit for bit under any
tile table; the PCG differs only in the rounding of its block-summed dot
products, so its solutions still meet the oracle's at 1e-10 (runs to 1e-13)
and its iteration counts at 1e-8 agree within one.  The autotuner's table
must be valid, be the one the solver keeps, describe the set-up levels, and
come back unchanged from its JSON cache.
"""
import json

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


def tile_class(n):
    return max(int(n), 1).bit_length() - 1


CASES = [
    P.laplace7(40),                                       # 64,000 cells: bricks, ragged tiles
    P.multipart_aniso(m=13, layout=(2, 1, 2), seed=3),    # couplings between parts
    P.var27(n=22, block=5, seed=2),                        # 27-point variable coefficients
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("prob", CASES, ids=[p.name for p in CASES])
def test_every_tile_form_gives_the_same_cycle(S, prob, prec):
    _, A = S.matrix_from_problem(prob)
    r = torch.as_tensor(P.SplitMix64(17).uniform_pm1(prob.n), device="cuda")

    def cycle(table):
        sv = S.Solver(precision=prec, flexible=prec)
        sv.set_tile_table(table)
        sv.setup(A)
        z = torch.zeros_like(r)
        sv.precondition(r, z)
        return sv, z

    ref_sv, ref = cycle(None)
    if prec == 0 and prob.n <= 30000:
        assert rel(ref.cpu().numpy(), O.vcycle(O.setup(prob), r.cpu().numpy())) <= 1e-12
    nl = ref_sv.num_levels()
    for k in (1, 2, 3, 4):
        for bricks in (0, S.TILE_BRICKS):
            sv, z = cycle([k | bricks] * S.TILE_CLASSES)
            assert torch.equal(z, ref), (k, bricks)
            for l in range(nl):
                cpt, b = sv.level_tile(l)
                assert cpt == k
                assert b == (1 if bricks and ref_sv.level_tile(l)[1] else 0), (l, k, bricks)


def test_mixed_table_by_size_class(S):
    """Different forms for different size classes in one hierarchy."""
    prob = P.laplace7(40)
    _, A = S.matrix_from_problem(prob)
    ref = S.Solver()
    ref.setup(A)
    table = [((c * 7) % 4 + 1) | (S.TILE_BRICKS if c % 2 else 0) for c in range(S.TILE_CLASSES)]
    sv = S.Solver()
    sv.set_tile_table(table)
    sv.setup(A)
    for l in range(sv.num_levels()):
        t = table[tile_class(sv.level_sizes(l)[0])]
        cpt, b = sv.level_tile(l)
        assert cpt == t & 7 and (b == 0 or t & S.TILE_BRICKS), l
    r = torch.as_tensor(P.SplitMix64(3).uniform_pm1(prob.n), device="cuda")
    z0, z1 = torch.zeros_like(r), torch.zeros_like(r)
    ref.precondition(r, z0)
    sv.precondition(r, z1)
    assert torch.equal(z0, z1)


def test_autotune_solver_and_cache(S, tmp_path):
    prob = P.multipart_aniso(m=16, layout=(2, 2, 2), seed=1)
    _, A = S.matrix_from_problem(prob)
    h = O.setup(prob)
    b = torch.as_tensor(prob.b[0], device="cuda")
    cache = str(tmp_path / "tiles.json")
    sv = S.Solver(precision=1, flexible=1, tol=1e-13, max_iter=400)
    sv.setup(A)
    table = sv.autotune(reps=5, cache=cache)
    assert len(table) == S.TILE_CLASSES and sv.tile_table() == table
    for t in table:
        assert t == 0 or 1 <= (t & ~S.TILE_BRICKS) <= 4
    for l in range(sv.num_levels()):
        t = table[tile_class(sv.level_sizes(l)[0])]
        if t:
            assert sv.level_tile(l)[0] == t & ~S.TILE_BRICKS
    x = torch.zeros_like(b)
    st = sv.solve(b, x)
    ref = O.pcg(h, prob.b[0], tol=1e-13, max_iter=400)
    assert st.converged and rel(x.cpu().numpy(), ref.x) <= 1e-10

    with open(cache) as f:
        assert json.load(f)[sv.tile_key()] == table
    sv2 = S.Solver(precision=1, flexible=1)
    sv2.setup(A)
    assert sv2.autotune(reps=5, cache=cache) == table and sv2.tile_table() == table
    x2 = torch.zeros_like(b)
    st2 = sv2.solve(b, x2)
    ref8 = O.pcg(h, prob.b[0], tol=1e-8)
    assert st2.converged and abs(st2.iterations - ref8.iterations) <= 1


def test_autotune_batch(S):
    probs = P.batched(nprob=6, nrhs=2, seed=21, pmax=3, emin=5, emax=14)
    mats = [S.matrix_from_problem(p) for p in probs]
    B = S.Batch([A for _, A in mats], precision=1, flexible=1)
    B.setup()
    table = B.autotune(reps=5)
    assert B.solver().tile_table() == table
    off = B.offsets()
    bh = np.zeros((2, off[-1]))
    for k, p in enumerate(probs):
        for j in range(2):
            bh[j, off[k]:off[k + 1]] = p.b[j]
    bt = torch.as_tensor(bh, device="cuda").contiguous()
    x = torch.zeros_like(bt)
    st = B.solve(bt, x, 2)
    for k, p in enumerate(probs):
        hk = O.setup(p)
        for j in range(2):
            ref = O.pcg(hk, p.b[j], tol=1e-8)
            assert st[j][k].converged and abs(st[j][k].iterations - ref.iterations) <= 1, (k, j)
