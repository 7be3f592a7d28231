"""Brute-force checker on assembled CSR matrices (test infrastructure only).

Independent of the stencil code in ``oracle.ssamg``: matrices are assembled
cell by cell with explicit loops, interpolation weights are recomputed from
the assembled rows (Section 3.2, Eq. prolEx, with the sign and boundary
readings stated in ``oracle.ssamg``), and Galerkin products are scipy sparse
triple products (Eq. galerkin).  Meant for grids of at most a few thousand
cells.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _cells(lo, hi):
    for k in range(lo[2], hi[2] + 1):
        for j in range(lo[1], hi[1] + 1):
            for i in range(lo[0], hi[0] + 1):
                yield (i, j, k)


class Numbering:
    """Global numbering of cells: parts in order, then k, j, i (i fastest)."""

    def __init__(self, los, his):
        self.los = [tuple(int(v) for v in x) for x in los]
        self.his = [tuple(int(v) for v in x) for x in his]
        self.start = [0]
        for lo, hi in zip(self.los, self.his):
            n = 1
            for d in range(3):
                n *= hi[d] - lo[d] + 1
            self.start.append(self.start[-1] + n)
        self.n = self.start[-1]
        self.part_of = np.zeros(self.n, np.int64)
        self.cell_of = [None] * self.n
        for p in range(len(self.los)):
            for t, c in enumerate(_cells(self.los[p], self.his[p])):
                self.part_of[self.start[p] + t] = p
                self.cell_of[self.start[p] + t] = c

    def inside(self, p, c):
        return all(self.los[p][d] <= c[d] <= self.his[p][d] for d in range(3))

    def index(self, p, c):
        lo, hi = self.los[p], self.his[p]
        nx = hi[0] - lo[0] + 1
        ny = hi[1] - lo[1] + 1
        return self.start[p] + ((c[2] - lo[2]) * ny + (c[1] - lo[1])) * nx + (c[0] - lo[0])


def _in_part(prob, p, c):
    """Cell c of part p's bounding box belongs to the part (one of its boxes)."""
    boxes = prob.part_boxes[p] if getattr(prob, "part_boxes", None) else None
    if boxes is None:
        return True
    return any(all(lo[d] <= c[d] <= hi[d] for d in range(3)) for lo, hi in boxes)


def assemble_problem(prob):
    """A = S + U of a problems.Problem as CSR, by loops over cells and entries
    (a part of several boxes over its bounding box: cells outside the boxes
    are rows of the identity, connections to them are dropped)."""
    num = Numbering([b[0] for b in prob.boxes], [b[1] for b in prob.boxes])
    rows, cols, vals = [], [], []
    for p in range(prob.nparts):
        lo, hi = prob.boxes[p]
        nx = hi[0] - lo[0] + 1
        ny = hi[1] - lo[1] + 1
        for c in _cells(lo, hi):
            loc = (c[0] - lo[0], c[1] - lo[1], c[2] - lo[2])
            if not _in_part(prob, p, c):
                rows.append(num.index(p, c))
                cols.append(num.index(p, c))
                vals.append(1.0)
                continue
            for e, o in enumerate(prob.offsets):
                nb = (c[0] + int(o[0]), c[1] + int(o[1]), c[2] + int(o[2]))
                if not num.inside(p, nb) or not _in_part(prob, p, nb):
                    continue
                co = prob.coef[p][e]
                v = float(co) if np.isscalar(co) else float(co[loc[2], loc[1], loc[0]])
                rows.append(num.index(p, c))
                cols.append(num.index(p, nb))
                vals.append(v)
    for t in range(prob.nnz_u):
        p, q = int(prob.u_part[t]), int(prob.u_nbor_part[t])
        rows.append(num.index(p, tuple(int(v) for v in prob.u_idx[t])))
        cols.append(num.index(q, tuple(int(v) for v in prob.u_nbor_idx[t])))
        vals.append(float(prob.u_val[t]))
    A = sp.coo_matrix((vals, (rows, cols)), shape=(num.n, num.n)).tocsr()
    A.sum_duplicates()
    return A, num


def assemble_level(lev):
    """A = S + U of an oracle Level as CSR, by loops over cells and entries."""
    num = Numbering(lev.lo, lev.hi)
    rows, cols, vals = [], [], []
    for p in range(lev.nparts):
        lo = num.los[p]
        for c in _cells(num.los[p], num.his[p]):
            loc = (c[0] - lo[0], c[1] - lo[1], c[2] - lo[2])
            for o, arr in lev.S[p].items():
                v = float(arr[loc[2], loc[1], loc[0]])
                nb = (c[0] + o[0], c[1] + o[1], c[2] + o[2])
                if not num.inside(p, nb):
                    if v != 0.0:
                        raise AssertionError(f"part {p} cell {c} entry {o} leaves the box with {v}")
                    continue
                rows.append(num.index(p, c))
                cols.append(num.index(p, nb))
                vals.append(v)
    rows += [int(r) for r in lev.u_row]
    cols += [int(c) for c in lev.u_col]
    vals += [float(v) for v in lev.u_val]
    A = sp.coo_matrix((vals, (rows, cols)), shape=(num.n, num.n)).tocsr()
    A.sum_duplicates()
    return A, num


def row_direction_bits(lev):
    bits = np.zeros(lev.n, np.int64)
    for r, b in zip(lev.u_row, lev.u_bits):
        bits[int(r)] |= int(b)
    return bits


def prolongation_brute(A, num, dstar, coarse_lo, coarse_hi, bits):
    """P as CSR (fine x coarse) from the assembled rows of A.

    For each fine cell f of a coarsened part (odd index along d*): sort the
    same-part entries of f's row by their offset along d*, form
    PW = -sum(-1 plane)/sum(0 plane), PE = -sum(+1 plane)/sum(0 plane), zero
    both if the denominator is ~0 or has the wrong sign, then apply the
    part-boundary fix using the direction bits of f's row.
    """
    cnum = Numbering(coarse_lo, coarse_hi)
    rows, cols, vals = [], [], []
    for g in range(num.n):
        p = int(num.part_of[g])
        c = num.cell_of[g]
        d = dstar[p]
        if d < 0:
            rows.append(g)
            cols.append(cnum.index(p, c))
            vals.append(1.0)
            continue
        if c[d] % 2 == 0:
            J = list(c)
            J[d] = c[d] // 2
            rows.append(g)
            cols.append(cnum.index(p, tuple(J)))
            vals.append(1.0)
            continue
        sw = se = den = 0.0
        diag = 0.0
        for t in range(A.indptr[g], A.indptr[g + 1]):
            col = int(A.indices[t])
            if int(num.part_of[col]) != p:
                continue
            cc = num.cell_of[col]
            off = cc[d] - c[d]
            v = float(A.data[t])
            if col == g:
                diag = v
            if off == -1:
                sw += v
            elif off == 1:
                se += v
            else:
                den += v
        if abs(den) > 1e-300 and np.sign(den) == np.sign(diag):
            pw, pe = -sw / den, -se / den
        else:
            pw = pe = 0.0
        if (bits[g] >> (2 * d)) & 1:
            pw, pe = 1.0, 0.0
        if (bits[g] >> (2 * d + 1)) & 1:
            pw, pe = 0.0, 1.0
        for J_d, w in (((c[d] - 1) // 2, pw), ((c[d] + 1) // 2, pe)):
            if coarse_lo[p][d] <= J_d <= coarse_hi[p][d]:
                J = list(c)
                J[d] = J_d
                rows.append(g)
                cols.append(cnum.index(p, tuple(J)))
                vals.append(w)
    return sp.coo_matrix((vals, (rows, cols)), shape=(num.n, cnum.n)).tocsr(), cnum


def galerkin(A, P):
    """P^T A P (Eq. galerkin) as a scipy sparse triple product."""
    return (P.T @ A @ P).tocsr()
