"""Bounded device waits end with an error status instead of hanging.

The grid barrier of the cooperative coarse-level kernel polls at most a
given number of times.  A self-test entry launches a small cooperative grid
whose barrier waits for arrivals that never come (a target above the grid
size): the blocks give up after a few hundred polls, the call reports
SSAMG_ERR_TIMEOUT, and the device and the solvers stay usable.  Nothing here
faults or traps; every wait returns.
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


def test_barrier_completes_when_every_block_arrives(S):
    for nb in (1, 2, 4):
        assert S.lib().ssamg_selftest_barrier(nb, 0, 1 << 16, None) == S.OK


def test_barrier_gives_up_at_its_cap_and_the_solver_still_works(S):
    stream = torch.cuda.current_stream().cuda_stream
    for nb in (1, 2):
        assert S.lib().ssamg_selftest_barrier(nb, 1, 300, stream) == S.ERR_TIMEOUT
        assert "poll cap" in S.last_error()
    # the context is intact: a cooperative-tail solver sets up and solves
    prob = P.multipart_aniso(m=6, layout=(2, 1, 1), seed=3)
    grid, A = S.matrix_from_problem(prob)
    sv = S.Solver(use_tail=1, tol=1e-10)
    sv.setup(A)
    b = torch.as_tensor(prob.b[0], device="cuda")
    x = torch.zeros_like(b)
    st = sv.solve(b, x)
    ref = O.pcg(O.setup(prob), prob.b[0], tol=1e-10)
    assert st.converged and abs(st.iterations - ref.iterations) <= 1
    assert np.abs(x.cpu().numpy() - ref.x).max() <= 1e-7 * np.abs(ref.x).max()
    assert S.lib().ssamg_selftest_barrier(2, 0, 1 << 16, stream) == S.OK
