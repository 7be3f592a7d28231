"""torch.autograd.Function over the SSAMG solve (the differentiation form).

x = A(a)^-1 b, where the level-0 operator A = S + U has per-cell stencil
coefficients a (entry-major, one row of N cells per stencil entry, parts in
order) and fixed inter-part couplings U.  The forward pass assembles A from
the coefficient tensor on the device, builds the hierarchy and runs
SSAMG-PCG.  The backward pass reuses that hierarchy for the adjoint solve
A^T lambda = dL/dx (A is symmetric for the operators this method targets,
so A^T = A and the same V-cycle applies) and maps lambda (x) x onto the
coefficients with the library's gradient kernel:
    dL/db = lambda,   dL/da_e(c) = -lambda_c x_{c + o_e}
(zero where c + o_e leaves the part's box, whose coefficients the assembly
drops).  Every step runs in libssamg.so; this module only marshals tensors.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence, Tuple

import torch

from . import ssamg as S


@dataclass
class Layout:
    """Index space and stencil of a semi-structured operator.

    ndim: 2 or 3; boxes: per part ((lo_x, lo_y, lo_z), (hi_x, hi_y, hi_z)),
    inclusive; offsets: per stencil entry (ox, oy, oz) in {-1, 0, 1};
    couplings: optional (part, idx, dir, nbor_part, nbor_idx, value) arrays
    in the form of Matrix.add_couplings (the U of A, not differentiated)."""
    ndim: int
    boxes: Sequence
    offsets: Sequence
    couplings: Optional[Tuple] = None
    params: dict = field(default_factory=dict)

    def part_sizes(self):
        out = []
        for lo, hi in self.boxes:
            n = 1
            for d in range(3):
                n *= hi[d] - lo[d] + 1
            out.append(n)
        return out


def _assemble(layout: Layout, coef: torch.Tensor):
    grid = S.Grid(layout.ndim, layout.boxes)
    A = S.Matrix(grid, layout.offsets)
    off = 0
    for p, n in enumerate(layout.part_sizes()):
        for e in range(len(layout.offsets)):
            A.set_box_values(p, e, coef[e, off:off + n])
        off += n
    if layout.couplings is not None:
        A.add_couplings(*layout.couplings)
    A.assemble()
    return grid, A


class StencilSolve(torch.autograd.Function):
    """x = A(coef)^-1 b, differentiable in coef (nentries x N, float64, CUDA)
    and b (N, float64, CUDA)."""

    @staticmethod
    def forward(ctx, coef: torch.Tensor, b: torch.Tensor, layout: Layout):
        if coef.dtype != torch.float64 or b.dtype != torch.float64:
            raise TypeError("coef and b must be float64")
        if not (coef.is_cuda and b.is_cuda):
            raise ValueError("coef and b must be CUDA tensors")
        coef = coef.detach().contiguous()
        b = b.detach().contiguous()
        grid, A = _assemble(layout, coef)
        sv = S.Solver(**layout.params)
        sv.setup(A)
        x = torch.zeros_like(b)
        sv.solve(b, x)
        ctx.keep = (grid, A, sv)
        ctx.nent = coef.shape[0]
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        (x,) = ctx.saved_tensors
        _, _, sv = ctx.keep
        lam = torch.zeros_like(x)
        sv.adjoint_solve(gx.detach().contiguous(), lam)
        dcoef = None
        if ctx.needs_input_grad[0]:
            dcoef = torch.empty(ctx.nent * x.numel(), dtype=x.dtype, device=x.device)
            sv.coef_gradient(lam, x, dcoef)
            dcoef = dcoef.view(ctx.nent, x.numel())
        return dcoef, (lam if ctx.needs_input_grad[1] else None), None


def stencil_solve(coef: torch.Tensor, b: torch.Tensor, layout: Layout) -> torch.Tensor:
    """Differentiable SSAMG-PCG solve (see StencilSolve)."""
    return StencilSolve.apply(coef, b, layout)
