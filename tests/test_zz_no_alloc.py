"""The allocation-free coupling-sum entry (ssamg_coupling_sums_noalloc).

Its block partials live in one static device array instead of solver memory,
so it is compared with the entry that reports the same sums from setup
(ssamg_spacings, level 0: bit for bit) and with the oracle (every level:
FP64 on both sides, only the summation order differs), on consecutive calls
that reuse the scratch, and inside a captured CUDA graph.
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


def _solver(S, prob):
    grid, A = S.matrix_from_problem(prob)
    sv = S.Solver()
    sv.setup(A)
    return grid, A, sv


def _sums(S, sv, level, nparts, stream=None):
    c = torch.full((nparts * 3,), float("nan"), dtype=torch.float64, device="cuda")
    sv.coupling_sums_noalloc(level, c, stream)
    return c


@pytest.mark.parametrize("prob", [
    P.multipart_aniso(m=11, layout=(2, 2, 2), seed=1),
    P.var27(n=13, block=3, seed=2),
    P.multipart_aniso(m=64, layout=(2, 2, 2), seed=1),   # level 0: 2048 blocks
], ids=["aniso8", "var27", "aniso8-64"])
def test_level0_matches_setup_entry_on_consecutive_calls(S, prob):
    _, _, sv = _solver(S, prob)
    nparts = len(prob.boxes)
    c_ref, _ = sv.spacings(nparts)
    for _ in range(2):
        c = _sums(S, sv, 0, nparts)
        torch.cuda.synchronize()
        assert np.array_equal(c.cpu().numpy().reshape(nparts, 3), c_ref)


def test_every_level_matches_oracle_and_scratch_reuse(S):
    prob = P.multipart_aniso(m=11, layout=(2, 2, 2), seed=1)
    h = O.setup(prob)
    _, _, sv = _solver(S, prob)
    nparts = len(prob.boxes)
    L = sv.num_levels()
    assert L == len(h.levels)
    first = []
    for l in range(L):
        c = _sums(S, sv, l, nparts).cpu().numpy().reshape(nparts, 3)
        ref = O.coupling_sums(h.levels[l])
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(c - ref).max() <= 1e-12 * scale, l
        first.append(c)
    # second pass in reverse order: each call overwrites the partials the
    # previous one left, so a slot read before it is written would show here
    for l in reversed(range(L)):
        c = _sums(S, sv, l, nparts).cpu().numpy().reshape(nparts, 3)
        assert np.array_equal(c, first[l]), l


def test_inside_captured_graph(S):
    prob = P.multipart_aniso(m=11, layout=(2, 2, 2), seed=3)
    _, _, sv = _solver(S, prob)
    nparts = len(prob.boxes)
    c_ref, _ = sv.spacings(nparts)
    out = torch.zeros(nparts * 3, dtype=torch.float64, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        sv.coupling_sums_noalloc(0, out, torch.cuda.current_stream())
    for _ in range(2):
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().reshape(nparts, 3), c_ref)


def test_rejects_bad_level(S):
    prob = P.laplace7(8)
    _, _, sv = _solver(S, prob)
    c = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        sv.coupling_sums_noalloc(sv.num_levels(), c)


def test_rejects_level_above_the_scratch(S):
    """A level whose launch needs more blocks than the static scratch holds
    is refused before anything is enqueued: one 257 x 256 x 256 part under a
    tile table of one cell per thread on its size class (2^24) gives
    16,842,752 / 256 = 65,792 blocks > 65,536."""
    prob = P.laplace7(1)
    prob = P.Problem(3, [((0, 0, 0), (256, 255, 255))], prob.offsets, prob.coef,
                     prob.u_part, prob.u_idx, prob.u_dir, prob.u_nbor_part, prob.u_nbor_idx,
                     prob.u_val, np.zeros((1, 1)), name="laplace7 257x256x256")
    grid, A = S.matrix_from_problem(prob)
    sv = S.Solver()
    table = [0] * S.TILE_CLASSES
    table[24] = 1
    sv.set_tile_table(table)
    sv.setup(A)
    assert sv.level_tile(0) == (1, 0)
    c = torch.full((3,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SsamgError) as e:
        sv.coupling_sums_noalloc(0, c)
    assert e.value.code == S.ERR_UNSUPPORTED
    msg = S.last_error()
    assert "65792" in msg and "65536" in msg, msg
    torch.cuda.synchronize()
    assert c.cpu().tolist() == [7.0, 7.0, 7.0]
    # level 1 (8,421,376 cells, 4 cells per thread) fits
    c1 = torch.zeros(3, dtype=torch.float64, device="cuda")
    sv.coupling_sums_noalloc(1, c1)
    torch.cuda.synchronize()
    assert np.isfinite(c1.cpu().numpy()).all()
