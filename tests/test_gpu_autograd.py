"""The torch.autograd.Function over the solve (differentiation form).

Gradients flow from a loss on x back to per-cell stencil coefficients (the
library's adjoint solve + coefficient-gradient kernel) and, through plain
torch operations written here, to the log-diffusivity g of the 7-point
harmonic-mean operator.  They are checked against the oracle's gradient
(adjoint and forward solves run to 1e-13 on both sides), against the
library's fused dL/dg kernel, and against central finite differences.
"""
import numpy as np
import pytest

import problems as P
from oracle import ssamg as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def AG(ssamg_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_14273_gb300 import autograd
    return autograd


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def diffusion_coef(g):
    """Entries [C, -x, +x, -y, +y, -z, +z] of the 7-point operator with face
    coefficient 2 k_c k_n / (k_c + k_n), k = exp(g), and k_c on each
    Dirichlet face (the operator of the differentiable workload)."""
    k = torch.exp(g)
    nz, ny, nx = g.shape
    diag = torch.zeros_like(k)
    rows = [None]
    for d, axis in ((0, 2), (1, 1), (2, 0)):
        for s in (-1, 1):
            kn = torch.roll(k, shifts=-s, dims=axis)
            idx = torch.arange(g.shape[axis], device=g.device)
            inside = (idx + s >= 0) & (idx + s < g.shape[axis])
            shape = [1, 1, 1]
            shape[axis] = -1
            inside = inside.view(shape).expand_as(k)
            t = 2.0 * k * kn / (k + kn)
            off = torch.where(inside, -t, torch.zeros_like(k))
            diag = diag + torch.where(inside, t, k)
            rows.append(off.reshape(-1))
    rows[0] = diag.reshape(-1)
    return torch.stack(rows)


def test_dg_through_autograd_matches_oracle_kernel_and_fd(AG):
    prob = P.diffusion_exp(n=10, seed=4, nfd=6)
    g0, xt, b = prob.extra["g"], prob.extra["x_t"], prob.b[0]
    nx = g0.shape[2]
    layout = AG.Layout(3, prob.boxes, prob.offsets, params=dict(tol=1e-13, max_iter=400))
    g = torch.tensor(g0, device="cuda", requires_grad=True)
    bt = torch.tensor(b, device="cuda", requires_grad=True)
    xtt = torch.as_tensor(xt, device="cuda")
    x = AG.stencil_solve(diffusion_coef(g), bt, layout)
    loss = 0.5 * ((x - xtt) ** 2).sum()
    loss.backward()

    h = O.setup(prob)
    xo = O.pcg(h, b, tol=1e-13).x
    lo = O.pcg(h, xo - xt, tol=1e-13).x
    ref = O.diffusion_exp_gradient(g0, lo, xo)
    assert rel(g.grad.cpu().numpy(), ref) <= 1e-9
    assert rel(bt.grad.cpu().numpy(), lo) <= 1e-9

    # the library's fused dL/dg kernel on the same adjoint state
    from paper_2205_14273_gb300 import ssamg as S
    grid, A = S.matrix_from_problem(prob)
    sv = S.Solver(tol=1e-13, max_iter=400)
    sv.setup(A)
    lam = torch.as_tensor(bt.grad.detach().cpu().numpy(), device="cuda")
    dg = torch.zeros_like(lam)
    sv.diffusion_exp_gradient(torch.as_tensor(g0.reshape(-1), device="cuda"), lam, x.detach(), dg)
    assert rel(g.grad.reshape(-1).cpu().numpy(), dg.cpu().numpy()) <= 1e-12

    def loss_at(gg):
        with torch.no_grad():
            xx = AG.stencil_solve(diffusion_coef(gg), bt.detach(), layout)
            return float(0.5 * ((xx - xtt) ** 2).sum())

    for c in prob.extra["fd_cells"][:3]:
        hstep = 1e-5
        e = torch.zeros(g0.size, dtype=torch.float64, device="cuda")
        e[c] = hstep
        e = e.view(g0.shape)
        gd = g.detach()
        fd = (loss_at(gd + e) - loss_at(gd - e)) / (2 * hstep)
        got = float(g.grad.reshape(-1)[c])
        assert abs(fd - got) <= 1e-6 * max(abs(fd), 1e-6), (c, fd, got)
    assert nx == 10


def test_coef_gradient_with_couplings_matches_oracle(AG):
    prob = P.multipart_aniso(m=6, layout=(2, 1, 2), seed=6)
    h = O.setup(prob)
    n = prob.n
    cells = h.levels[0].offsets()
    rows = []
    for e in range(len(prob.offsets)):
        row = np.zeros(n)
        for p in range(prob.nparts):
            c = prob.coef[p][e]
            row[cells[p]:cells[p + 1]] = c if np.isscalar(c) else np.asarray(c).ravel()
        rows.append(row)
    coef = torch.tensor(np.stack(rows), device="cuda", requires_grad=True)
    w = P.SplitMix64(5).uniform_pm1(n)
    layout = AG.Layout(prob.ndim, prob.boxes, prob.offsets,
                       couplings=(prob.u_part, prob.u_idx, prob.u_dir, prob.u_nbor_part,
                                  prob.u_nbor_idx, prob.u_val),
                       params=dict(tol=1e-13, max_iter=400))
    b = torch.as_tensor(prob.b[0], device="cuda")
    x = AG.stencil_solve(coef, b, layout)
    (x * torch.as_tensor(w, device="cuda")).sum().backward()

    xo = O.pcg(h, prob.b[0], tol=1e-13).x
    lo = O.pcg(h, w, tol=1e-13).x
    assert rel(x.detach().cpu().numpy(), xo) <= 1e-10
    ref = O.coef_gradient(h.levels[0], lo, xo)
    got = coef.grad.cpu().numpy()
    for e, o in enumerate(prob.offsets):
        o = tuple(int(v) for v in o)
        for p in range(prob.nparts):
            assert rel(got[e, cells[p]:cells[p + 1]], ref[p][o].reshape(-1)) <= 1e-9


def test_diffusion_gradient_refuses_other_grids(ssamg_lib):
    """The dL/dg kernel differentiates one box with the 7-point faces: a
    two-part solver and a 27-point stencil are refused (SSAMG_ERR_UNSUPPORTED)
    and the output is left as it was; wrong vectors are refused by the
    binding before the call."""
    S = ssamg_lib
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for prob in (P.multipart_aniso(m=4, layout=(2, 1, 1), seed=2), P.var27(n=6, block=2, seed=2)):
        grid, A = S.matrix_from_problem(prob)
        sv = S.Solver()
        sv.setup(A)
        n = prob.n
        v = torch.ones(n, dtype=torch.float64, device="cuda")
        dg = torch.full((n,), 3.0, dtype=torch.float64, device="cuda")
        with pytest.raises(S.SsamgError) as e:
            sv.diffusion_exp_gradient(v, v, v, dg)
        assert e.value.code == S.ERR_UNSUPPORTED
        torch.cuda.synchronize()
        assert bool((dg == 3.0).all())
    prob = P.diffusion_exp(n=6, seed=4, nfd=2)
    grid, A = S.matrix_from_problem(prob)
    sv = S.Solver()
    sv.setup(A)
    n = prob.n
    v = torch.ones(n, dtype=torch.float64, device="cuda")
    for bad in (torch.ones(n, dtype=torch.float32, device="cuda"),
                torch.ones(n - 1, dtype=torch.float64, device="cuda")):
        with pytest.raises(ValueError):
            sv.diffusion_exp_gradient(v, v, v, bad)
        with pytest.raises(ValueError):
            sv.solve(bad, torch.zeros(n, dtype=torch.float64, device="cuda"))
