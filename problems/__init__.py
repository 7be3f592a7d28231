"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only *describes* linear systems (grid boxes, stencil coefficients,
inter-part couplings, right-hand sides).  It contains none of the SSAMG
arithmetic: no coarsening, interpolation, Galerkin products, relaxation or
Krylov steps.  Both sides receive the same arrays produced here.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the n-th output of seed s is
mix(s + n * 0x9E3779B97F4A7C15) with the published 64-bit finaliser.  Uniform
[0,1) draws take the top 53 bits times 2**-53; log-uniform(a,b) is
exp(ln a + u (ln b - ln a)); normals use Box-Muller on consecutive pairs.

The workloads mirror the paper's test problems (Section 4: 3-D finite
difference diffusion on cell-centred boxes with Dirichlet boundaries, Eq.
stencilA; anisotropic parts as in test case 2) at the sizes the GB300 build
targets:

  laplace7        one part, constant 7-point Laplacian (6, -1 x 6)
  multipart_aniso parts in a block layout, per-part anisotropy, inter-part
                  couplings by harmonic means (variable diagonal)
  var27           one part, 27-point variable-coefficient diffusion with
                  block-constant coefficients
  batched         many independent multi-part problems chained along x
  diffusion_exp   one part, 7-point diffusion with kappa = exp(g), g smoothed
                  Gaussian noise (differentiable workload)
  three_point     three cubes around a common k edge, couplings across
                  rotated index maps (test case 3, non-Cartesian)
  samr            a coarse part with ghost unknowns under a refined patch of
                  twice the resolution (test case 4, SAMR)
  multibox        an L-shaped part of two boxes around a cube part filling
                  its notch (a part of several boxes, Section 2)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple, Union

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64 stream: output n (1-based) = mix(seed + n*golden)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.pos = 0  # number of outputs consumed so far

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            idx = np.arange(self.pos + 1, self.pos + 1 + n, dtype=np.uint64)
            z = self.seed + idx * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        self.pos += n
        return z

    def uniform(self, n: int) -> np.ndarray:
        """n draws in [0, 1): top 53 bits x 2**-53."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def uniform_pm1(self, n: int) -> np.ndarray:
        return 2.0 * self.uniform(n) - 1.0

    def log_uniform(self, n: int, a: float, b: float) -> np.ndarray:
        la, lb = math.log(a), math.log(b)
        return np.exp(la + self.uniform(n) * (lb - la))

    def int_range(self, n: int, lo: int, hi: int) -> np.ndarray:
        """n integers uniform in {lo, ..., hi} (inclusive)."""
        return lo + np.floor(self.uniform(n) * (hi - lo + 1)).astype(np.int64)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by Box-Muller on consecutive uniform pairs."""
        m = (n + 1) // 2
        u = self.uniform(2 * m)
        u1, u2 = u[0::2], u[1::2]
        rad = np.sqrt(-2.0 * np.log1p(-u1))
        z = np.empty(2 * m)
        z[0::2] = rad * np.cos(2.0 * math.pi * u2)
        z[1::2] = rad * np.sin(2.0 * math.pi * u2)
        return z[:n]


# ---------------------------------------------------------------------------
# Problem description (the semi-structured matrix A = S + U and a RHS)
# ---------------------------------------------------------------------------

Coef = Union[float, np.ndarray]


@dataclass
class Problem:
    """A semi-structured linear system A x = b (Section 2: grid, stencil, graph).

    boxes[p] = (lo, hi): inclusive cell-centred corners of part p (3 ints each;
        unused dimensions have lo = hi).
    offsets: (k, 3) stencil offsets shared by all parts, entries in {-1,0,1}.
    coef[p][e]: a float (entry constant over the part) or an array of shape
        (nz, ny, nx) (i fastest in memory).  Entries pointing outside the part
        box are ignored (the structured matrix S has no such connections).
    Couplings (the unstructured matrix U), one entry per row:
        u_part, u_idx (local cell of the row), u_dir (offset that leaves the
        part, or 0,0,0), u_nbor_part, u_nbor_idx (local cell of the column),
        u_val.  Indices are absolute (in the part's index space).
    b: (nrhs, N) right-hand sides, parts in order, i fastest.
    """

    ndim: int
    boxes: List[Tuple[Tuple[int, int, int], Tuple[int, int, int]]]
    offsets: np.ndarray
    coef: List[List[Coef]]
    u_part: np.ndarray
    u_idx: np.ndarray
    u_dir: np.ndarray
    u_nbor_part: np.ndarray
    u_nbor_idx: np.ndarray
    u_val: np.ndarray
    b: np.ndarray
    name: str = ""
    extra: dict = field(default_factory=dict)
    # parts made of several boxes (Section 2): part_boxes[p] lists the boxes
    # (lo, hi) of part p, boxes[p] being their bounding box; None (or None
    # for a part) means the part is its bounding box.  Coefficient arrays and
    # right-hand sides cover the bounding box; cells outside the part's boxes
    # carry no connections (their values are ignored).
    part_boxes: Optional[List[Optional[List[Tuple[Tuple[int, int, int], Tuple[int, int, int]]]]]] = None

    @property
    def nparts(self) -> int:
        return len(self.boxes)

    def shape(self, p: int) -> Tuple[int, int, int]:
        lo, hi = self.boxes[p]
        return (hi[2] - lo[2] + 1, hi[1] - lo[1] + 1, hi[0] - lo[0] + 1)

    def part_sizes(self) -> List[int]:
        return [int(np.prod(self.shape(p))) for p in range(self.nparts)]

    @property
    def n(self) -> int:
        return int(sum(self.part_sizes()))

    @property
    def nnz_u(self) -> int:
        return int(len(self.u_val))


def _empty_u():
    return (np.zeros(0, np.int32), np.zeros((0, 3), np.int32), np.zeros((0, 3), np.int32),
            np.zeros(0, np.int32), np.zeros((0, 3), np.int32), np.zeros(0, np.float64))


STENCIL7 = np.array([(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0),
                     (0, 0, -1), (0, 0, 1)], dtype=np.int32)

STENCIL27 = np.array([(0, 0, 0)] + [(i, j, k) for k in (-1, 0, 1) for j in (-1, 0, 1)
                                    for i in (-1, 0, 1) if (i, j, k) != (0, 0, 0)],
                     dtype=np.int32)


def laplace7(n: int = 32, seed: int = 0, nrhs: int = 1) -> Problem:
    """One part [0,n-1]^3, constant 7-point stencil (6, -1 x 6); Dirichlet
    boundaries eliminated (Eq. stencilA with alpha = beta = gamma = 1)."""
    rng = SplitMix64(seed)
    coef = [[6.0] + [-1.0] * 6]
    b = rng.uniform_pm1(nrhs * n ** 3).reshape(nrhs, n ** 3)
    return Problem(3, [((0, 0, 0), (n - 1, n - 1, n - 1))], STENCIL7.copy(), coef,
                   *_empty_u(), b, name=f"laplace7 {n}^3")


def _harmonic(a, b):
    return 2.0 * a * b / (a + b)


def multipart_aniso(m: int = 64, layout: Sequence[int] = (2, 2, 2), seed: int = 1,
                    amin: float = 1e-3, amax: float = 1.0, nrhs: int = 1) -> Problem:
    """Parts of m^3 cells in a block layout (part index px + Lx*(py + Ly*pz)).

    Per part, (a_x, a_y, a_z) ~ log-uniform[amin, amax] (drawn part-major).
    Off-diagonal stencil entries are the constants -a_d.  Facing cells of
    neighbouring parts are coupled (both directions) by -2 a_p a_q / (a_p + a_q)
    with a_p, a_q the parts' coefficients normal to the interface.  The
    diagonal is the sum of |off-diagonals| of S and U plus a_d for every
    Dirichlet face of the cell, i.e. 2(a_x+a_y+a_z) away from interfaces.
    """
    rng = SplitMix64(seed)
    Lx, Ly, Lz = layout
    npart = Lx * Ly * Lz
    a = rng.log_uniform(3 * npart, amin, amax).reshape(npart, 3)
    pos = {}
    for p in range(npart):
        px, py, pz = p % Lx, (p // Lx) % Ly, p // (Lx * Ly)
        pos[(px, py, pz)] = p
    boxes = [((0, 0, 0), (m - 1, m - 1, m - 1)) for _ in range(npart)]
    coef = []
    up, ui, ud, uq, uj, uv = [], [], [], [], [], []
    g = np.arange(m)
    kk, jj, ii = np.meshgrid(g, g, g, indexing="ij")
    for p in range(npart):
        px, py, pz = p % Lx, (p // Lx) % Ly, p // (Lx * Ly)
        ppos = (px, py, pz)
        diag = np.full((m, m, m), 2.0 * a[p].sum())
        for d in range(3):
            for s in (-1, 1):
                npos = list(ppos)
                npos[d] += s
                q = pos.get(tuple(npos))
                if q is None:
                    continue
                u = -_harmonic(a[p, d], a[q, d])
                face = m - 1 if s > 0 else 0
                # cells of p on this face; the matching cell of q sits on its opposite face
                sl = [slice(None)] * 3
                sl[2 - d] = face
                diag[tuple(sl)] += abs(u) - a[p, d]
                cells = np.stack([ii[tuple(sl)].ravel(), jj[tuple(sl)].ravel(),
                                  kk[tuple(sl)].ravel()], axis=1)
                nb = cells.copy()
                nb[:, d] = (m - 1) - face
                dvec = np.zeros(3, np.int32)
                dvec[d] = s
                up.append(np.full(len(cells), p))
                ui.append(cells)
                ud.append(np.tile(dvec, (len(cells), 1)))
                uq.append(np.full(len(cells), q))
                uj.append(nb)
                uv.append(np.full(len(cells), u))
        coef.append([diag, -a[p, 0], -a[p, 0], -a[p, 1], -a[p, 1], -a[p, 2], -a[p, 2]])
    N = npart * m ** 3
    b = rng.uniform_pm1(nrhs * N).reshape(nrhs, N)
    cat = lambda xs, dt, shape: (np.concatenate(xs).astype(dt) if xs else np.zeros(shape, dt))
    return Problem(3, boxes, STENCIL7.copy(), coef,
                   cat(up, np.int32, 0), cat(ui, np.int32, (0, 3)), cat(ud, np.int32, (0, 3)),
                   cat(uq, np.int32, 0), cat(uj, np.int32, (0, 3)), cat(uv, np.float64, 0),
                   b, name=f"multipart_aniso {npart}x{m}^3", extra={"a": a})


def var27(n: int = 256, block: int = 8, seed: int = 2, kmin: float = 1e-4,
          kmax: float = 1e4, nrhs: int = 1) -> Problem:
    """One part [0,n-1]^3 with a 27-point variable-coefficient stencil.

    kappa ~ log-uniform[kmin, kmax], constant on block^3 blocks (block order
    i fastest).  Off-diagonal (c, c+o) = -2 k_c k_n / (k_c + k_n) for all 26
    neighbours inside the box; diagonal = sum |off| + k_c per missing
    neighbour (SPD, diagonally dominant).
    """
    rng = SplitMix64(seed)
    nb = -(-n // block)
    kb = rng.log_uniform(nb ** 3, kmin, kmax).reshape(nb, nb, nb)
    idx = np.arange(n) // block
    kap = kb[idx][:, idx][:, :, idx]  # (z, y, x)
    coef = [None] * 27
    diag = np.zeros((n, n, n))
    for e in range(1, 27):
        ox, oy, oz = (int(v) for v in STENCIL27[e])
        off = np.zeros((n, n, n))
        src = [slice(max(0, -o), n - max(0, o)) for o in (oz, oy, ox)]
        dst = [slice(max(0, o), n - max(0, -o)) for o in (oz, oy, ox)]
        kc = kap[tuple(src)]
        kn = kap[tuple(dst)]
        off[tuple(src)] = -_harmonic(kc, kn)
        inside = np.zeros((n, n, n), bool)
        inside[tuple(src)] = True
        diag += np.where(inside, -off, kap)
        coef[e] = off
    coef[0] = diag
    b = rng.uniform_pm1(nrhs * n ** 3).reshape(nrhs, n ** 3)
    return Problem(3, [((0, 0, 0), (n - 1, n - 1, n - 1))], STENCIL27.copy(), [coef],
                   *_empty_u(), b, name=f"var27 {n}^3", extra={"kappa_block": kb})


def chain_aniso(edges: Sequence[int], a: np.ndarray, rng: SplitMix64, nrhs: int) -> Problem:
    """Parts with cube edges `edges` chained along x, aligned at j = k = 0.

    Couplings (harmonic means of the x coefficients) exist on the overlap of
    adjacent x faces; the rest of every face is Dirichlet.  Coefficients as in
    multipart_aniso with a[p] = (a_x, a_y, a_z).
    """
    npart = len(edges)
    boxes = [((0, 0, 0), (e - 1, e - 1, e - 1)) for e in edges]
    coef = []
    up, ui, ud, uq, uj, uv = [], [], [], [], [], []
    for p, m in enumerate(edges):
        diag = np.full((m, m, m), 2.0 * a[p].sum())
        for s in (-1, 1):
            q = p + s
            if q < 0 or q >= npart:
                continue
            mq = edges[q]
            ov = min(m, mq)
            u = -_harmonic(a[p, 0], a[q, 0])
            face = m - 1 if s > 0 else 0
            nface = 0 if s > 0 else mq - 1
            diag[:ov, :ov, face] += abs(u) - a[p, 0]
            kk, jj = np.meshgrid(np.arange(ov), np.arange(ov), indexing="ij")
            cnt = ov * ov
            cells = np.stack([np.full(cnt, face), jj.ravel(), kk.ravel()], axis=1)
            nbc = np.stack([np.full(cnt, nface), jj.ravel(), kk.ravel()], axis=1)
            up.append(np.full(cnt, p))
            ui.append(cells)
            ud.append(np.tile(np.array([s, 0, 0]), (cnt, 1)))
            uq.append(np.full(cnt, q))
            uj.append(nbc)
            uv.append(np.full(cnt, u))
        coef.append([diag, -a[p, 0], -a[p, 0], -a[p, 1], -a[p, 1], -a[p, 2], -a[p, 2]])
    N = int(sum(e ** 3 for e in edges))
    b = rng.uniform_pm1(nrhs * N).reshape(nrhs, N)
    cat = lambda xs, dt, shape: (np.concatenate(xs).astype(dt) if xs else np.zeros(shape, dt))
    return Problem(3, boxes, STENCIL7.copy(), coef,
                   cat(up, np.int32, 0), cat(ui, np.int32, (0, 3)), cat(ud, np.int32, (0, 3)),
                   cat(uq, np.int32, 0), cat(uj, np.int32, (0, 3)), cat(uv, np.float64, 0),
                   b, name=f"chain {list(edges)}", extra={"a": a})


def batched(nprob: int = 64, nrhs: int = 4, seed: int = 3, pmin: int = 1, pmax: int = 8,
            emin: int = 16, emax: int = 96) -> List[Problem]:
    """Independent multi-part problems of uneven sizes, all from one stream.

    Per problem, in draw order: number of parts ~ U{pmin..pmax}; each part's
    cube edge ~ U{emin..emax}; per part (a_x, a_y, a_z) ~ log-uniform[1e-3, 1];
    then nrhs right-hand sides ~ U[-1, 1].
    """
    rng = SplitMix64(seed)
    out = []
    for _ in range(nprob):
        npart = int(rng.int_range(1, pmin, pmax)[0])
        edges = [int(v) for v in rng.int_range(npart, emin, emax)]
        a = rng.log_uniform(3 * npart, 1e-3, 1.0).reshape(npart, 3)
        out.append(chain_aniso(edges, a, rng, nrhs))
    return out


def box_mean_truncated(g: np.ndarray, w: int) -> np.ndarray:
    """Mean over the (2w+1)^3 window around each cell, truncated at the edges."""
    out = g.copy()
    cnt = np.ones_like(g)
    for ax in range(3):
        n = g.shape[ax]
        cs = np.cumsum(np.concatenate([np.zeros_like(np.take(out, [0], axis=ax)), out], axis=ax), axis=ax)
        cc = np.cumsum(np.concatenate([np.zeros_like(np.take(cnt, [0], axis=ax)), cnt], axis=ax), axis=ax)
        lo = np.clip(np.arange(n) - w, 0, n)
        hi = np.clip(np.arange(n) + w + 1, 0, n)
        out = np.take(cs, hi, axis=ax) - np.take(cs, lo, axis=ax)
        cnt = np.take(cc, hi, axis=ax) - np.take(cc, lo, axis=ax)
    return out / cnt


def diffusion_exp(n: int = 128, seed: int = 4, nfd: int = 32, smooth: int = 2) -> Problem:
    """One part [0,n-1]^3, 7-point diffusion with kappa = exp(g).

    g: i.i.d. N(0,1) per cell, then the mean over a (2*smooth+1)^3 window
    truncated at the domain edge, then divided by its sample std.  Off-
    diagonals -2 k_c k_n/(k_c+k_n); diagonal = sum |off| + k_c per Dirichlet
    face.  Then x_t ~ U[-1,1], b ~ U[-1,1], and nfd finite-difference probe
    cells ~ U{0..N-1}, in that draw order.
    """
    rng = SplitMix64(seed)
    N = n ** 3
    g = rng.normal(N).reshape(n, n, n)
    g = box_mean_truncated(g, smooth)
    g = g / g.std()
    x_t = rng.uniform_pm1(N)
    b = rng.uniform_pm1(N).reshape(1, N)
    fd_cells = rng.int_range(nfd, 0, N - 1)
    prob = diffusion_from_g(g, b)
    prob.extra.update({"g": g, "x_t": x_t, "fd_cells": fd_cells})
    prob.name = f"diffusion_exp {n}^3"
    return prob


def diffusion_from_g(g: np.ndarray, b: np.ndarray) -> Problem:
    """The 7-point harmonic-mean diffusion operator for kappa = exp(g)."""
    nz, ny, nx = g.shape
    kap = np.exp(g)
    coef = [None] * 7
    diag = np.zeros_like(kap)
    for e in range(1, 7):
        ox, oy, oz = (int(v) for v in STENCIL7[e])
        off = np.zeros_like(kap)
        shp = (nz, ny, nx)
        src = tuple(slice(max(0, -o), s - max(0, o)) for o, s in zip((oz, oy, ox), shp))
        dst = tuple(slice(max(0, o), s - max(0, -o)) for o, s in zip((oz, oy, ox), shp))
        off[src] = -_harmonic(kap[src], kap[dst])
        inside = np.zeros(shp, bool)
        inside[src] = True
        diag += np.where(inside, -off, kap)
        coef[e] = off
    coef[0] = diag
    return Problem(3, [((0, 0, 0), (nx - 1, ny - 1, nz - 1))], STENCIL7.copy(), [coef],
                   *_empty_u(), np.asarray(b, np.float64).reshape(-1, nx * ny * nz),
                   extra={"g": g})


def three_point(m: int = 160, seed: int = 5, nrhs: int = 1) -> Problem:
    """Three parts of m^3 cells around a common edge along k (test case 3).

    Each part is [0,m-1]^3 in its own index space with the isotropic 7-point
    Laplacian (6, -1 x 6).  The east face of part p (i = m-1) touches the
    north face of part q = p+1 mod 3 (j = m-1), the shared edge being each
    part's (i, j) = (m-1, m-1) corner: cell (m-1, t, k) of p and cell
    (t, m-1, k) of q are coupled by -1 both ways, so an east connection of p
    is a north connection of q (the index maps are not Cartesian).  West,
    south, bottom and top faces are Dirichlet (eliminated), so the diagonal
    is 6 everywhere.
    """
    rng = SplitMix64(seed)
    boxes = [((0, 0, 0), (m - 1, m - 1, m - 1)) for _ in range(3)]
    coef = [[6.0] + [-1.0] * 6 for _ in range(3)]
    kk, tt = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    kk, tt = kk.ravel(), tt.ravel()
    cnt = m * m
    east = np.stack([np.full(cnt, m - 1), tt, kk], axis=1)   # (m-1, t, k) of p
    north = np.stack([tt, np.full(cnt, m - 1), kk], axis=1)  # (t, m-1, k) of q
    up, ui, ud, uq, uj = [], [], [], [], []
    for p in range(3):
        q = (p + 1) % 3
        up += [np.full(cnt, p), np.full(cnt, q)]
        ui += [east, north]
        ud += [np.tile(np.array([1, 0, 0]), (cnt, 1)), np.tile(np.array([0, 1, 0]), (cnt, 1))]
        uq += [np.full(cnt, q), np.full(cnt, p)]
        uj += [north, east]
    uv = np.full(6 * cnt, -1.0)
    N = 3 * m ** 3
    b = rng.uniform_pm1(nrhs * N).reshape(nrhs, N)
    return Problem(3, boxes, STENCIL7.copy(), coef,
                   np.concatenate(up).astype(np.int32), np.concatenate(ui).astype(np.int32),
                   np.concatenate(ud).astype(np.int32), np.concatenate(uq).astype(np.int32),
                   np.concatenate(uj).astype(np.int32), uv, b, name=f"three_point 3x{m}^3")


def samr(m: int = 128, seed: int = 6, nrhs: int = 1, cf: float = 2.0 / 3.0) -> Problem:
    """A structured AMR grid of two parts with m^3 cells each (test case 4).

    Part 0, [0,m-1]^3, is the coarse grid; its cells in the central cube
    G = [m/4, 3m/4-1]^3 are ghost unknowns (diagonal 1, no off-diagonals, zero
    right-hand side).  Part 1 refines G by two: [m/2, 3m/2-1]^3 in its own
    index space, fine cell f under coarse cell f // 2.  Both parts carry the
    7-point Laplacian (-1 between neighbouring cells of the same part, none
    into or out of G).  Across the patch boundary each fine face cell is
    coupled to the coarse cell beside its parent, and each such coarse cell
    to the four fine cells facing it, by -cf (cf = 2/3) both ways.  Rows of
    the fine part leave its box through a face; rows of the coarse part lie
    inside its box beside G (direction 0, 0, 0).  Diagonals: the sum of the
    row's |off-diagonals| plus 1 per Dirichlet face of the outer box.
    """
    assert m % 4 == 0
    rng = SplitMix64(seed)
    g0, g1 = m // 4, 3 * m // 4 - 1
    f0, f1 = 2 * g0, 2 * g1 + 1
    boxes = [((0, 0, 0), (m - 1, m - 1, m - 1)), ((f0, f0, f0), (f1, f1, f1))]
    ax = np.arange(m)
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    ghost = ((xx >= g0) & (xx <= g1) & (yy >= g0) & (yy <= g1) & (zz >= g0) & (zz <= g1))
    # coarse part: -1 between non-ghost neighbours inside the box
    cdiag = np.zeros((m, m, m))
    ccoef = []
    for o in STENCIL7[1:]:
        ox, oy, oz = (int(v) for v in o)
        nx, ny, nz = xx + ox, yy + oy, zz + oz
        inb = (nx >= 0) & (nx < m) & (ny >= 0) & (ny < m) & (nz >= 0) & (nz < m)
        ng = np.zeros_like(ghost)
        ng[inb] = ghost[nz[inb], ny[inb], nx[inb]]
        off = np.where(inb & ~ghost & ~ng, -1.0, 0.0)
        cdiag += np.where(inb, -off, 1.0)  # a Dirichlet face adds 1
        cdiag += np.where(inb & ~ghost & ng, 4 * cf, 0.0)  # four fine cells across
        ccoef.append(off)
    cdiag = np.where(ghost, 1.0, cdiag)
    # fine part: -1 inside its box; every face is coupled to the coarse part
    fdiag = np.full((m, m, m), 6.0)
    for d in range(3):
        for side in (0, m - 1):
            sl = [slice(None)] * 3
            sl[2 - d] = side
            fdiag[tuple(sl)] += cf - 1.0
    up, ui, ud, uq, uj = [], [], [], [], []
    fa = np.arange(f0, f1 + 1)
    ca = np.arange(g0, g1 + 1)
    for d in range(3):
        for s, fface, cnb in ((-1, f0, g0 - 1), (1, f1, g1 + 1)):
            # fine rows: face cells, column = the coarse cell beside the parent
            u1, u2 = np.meshgrid(fa, fa, indexing="ij")
            u1, u2 = u1.ravel(), u2.ravel()
            fc = np.zeros((len(u1), 3), np.int64)
            fc[:, d] = fface
            fc[:, (d + 1) % 3] = u1
            fc[:, (d + 2) % 3] = u2
            cc = fc // 2
            cc[:, d] = cnb
            dv = np.zeros((len(u1), 3), np.int64)
            dv[:, d] = s
            up.append(np.full(len(u1), 1))
            ui.append(fc)
            ud.append(dv)
            uq.append(np.full(len(u1), 0))
            uj.append(cc)
            # coarse rows: the cells beside G, each to its four fine cells
            up.append(np.full(len(u1), 0))
            ui.append(cc)
            ud.append(np.zeros((len(u1), 3), np.int64))
            uq.append(np.full(len(u1), 1))
            uj.append(fc)
    nu = sum(len(x) for x in up)
    N = 2 * m ** 3
    b = rng.uniform_pm1(nrhs * N).reshape(nrhs, N)
    b[:, :m ** 3] *= ~ghost.ravel()
    coef = [[cdiag] + ccoef, [fdiag] + [-1.0] * 6]
    return Problem(3, boxes, STENCIL7.copy(), coef,
                   np.concatenate(up).astype(np.int32), np.concatenate(ui).astype(np.int32),
                   np.concatenate(ud).astype(np.int32), np.concatenate(uq).astype(np.int32),
                   np.concatenate(uj).astype(np.int32), np.full(nu, -cf), b,
                   name=f"samr 2x{m}^3", extra={"ghost": ghost})


def box_mask(shape_zyx, lo, boxes) -> np.ndarray:
    """Cells of a bounding box (shape (nz, ny, nx), corner lo) that lie in
    any of `boxes`."""
    nz, ny, nx = shape_zyx
    zz, yy, xx = np.meshgrid(np.arange(nz) + lo[2], np.arange(ny) + lo[1],
                             np.arange(nx) + lo[0], indexing="ij")
    m = np.zeros(shape_zyx, bool)
    for blo, bhi in boxes:
        m |= ((xx >= blo[0]) & (xx <= bhi[0]) & (yy >= blo[1]) & (yy <= bhi[1]) &
              (zz >= blo[2]) & (zz <= bhi[2]))
    return m


def multibox(m: int = 64, seed: int = 7, nrhs: int = 1) -> Problem:
    """Two parts (Section 2, a part of several boxes, as Part 4 of Fig. ssgrid).

    Part 0 is L-shaped: boxes [0, 2m-1] x [0, m-1] x [0, m-1] and
    [0, m-1] x [m, 2m-1] x [0, m-1], bounding box [0, 2m-1]^2 x [0, m-1]; its
    notch [m, 2m-1]^2 x [0, m-1] is filled by part 1, [0, m-1]^3 in its own
    index space (cell (i, j, k) of part 1 sits at (m + i, m + j, k) of part
    0's index space).  Both parts carry the 7-point Laplacian (6, -1 x 6)
    between cells of the same part; facing cells of the two parts are coupled
    by -1 both ways, the rows of part 0 leaving it through +x (the notch's
    west face) or +y (its south face) from inside its bounding box.  Other
    faces are Dirichlet: the diagonal stays 6.
    """
    rng = SplitMix64(seed)
    b0 = [((0, 0, 0), (2 * m - 1, m - 1, m - 1)), ((0, m, 0), (m - 1, 2 * m - 1, m - 1))]
    boxes = [((0, 0, 0), (2 * m - 1, 2 * m - 1, m - 1)), ((0, 0, 0), (m - 1, m - 1, m - 1))]
    up, ui, ud, uq, uj = [], [], [], [], []
    t, k = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    t, k = t.ravel(), k.ravel()
    cnt = m * m
    for d in (0, 1):
        # part 0 cells just outside the notch along d, part 1's cells on its face
        c0 = np.zeros((cnt, 3), np.int64)
        c0[:, d] = m - 1
        c0[:, 1 - d] = m + t
        c0[:, 2] = k
        c1 = np.zeros((cnt, 3), np.int64)
        c1[:, d] = 0
        c1[:, 1 - d] = t
        c1[:, 2] = k
        dv = np.zeros((cnt, 3), np.int64)
        dv[:, d] = 1
        up += [np.zeros(cnt), np.ones(cnt)]
        ui += [c0, c1]
        ud += [dv, -dv]
        uq += [np.ones(cnt), np.zeros(cnt)]
        uj += [c1, c0]
    N0 = 4 * m ** 3
    N = N0 + m ** 3
    b = rng.uniform_pm1(nrhs * N).reshape(nrhs, N)
    act = box_mask((m, 2 * m, 2 * m), (0, 0, 0), b0).ravel()
    b[:, :N0] *= act
    coef = [[6.0] + [-1.0] * 6, [6.0] + [-1.0] * 6]
    return Problem(3, boxes, STENCIL7.copy(), coef,
                   np.concatenate(up).astype(np.int32), np.concatenate(ui).astype(np.int32),
                   np.concatenate(ud).astype(np.int32), np.concatenate(uq).astype(np.int32),
                   np.concatenate(uj).astype(np.int32), np.full(4 * cnt, -1.0), b,
                   name=f"multibox L(2 boxes)+{m}^3", part_boxes=[b0, None])


def config(k: int, small: bool = False) -> Union[Problem, List[Problem]]:
    """The workloads at full size (small=False) or at a size the oracle
    finishes in seconds (small=True) with the same structure and seeds:
    0-4 as listed above, 5 the three-point intersection (3 x 160^3) and 6 the
    SAMR grid (2 x 128^3) of the paper's test cases 3 and 4, 7 a part of two
    boxes (an L of 3 x 96^3 cells) around a 96^3 part."""
    if k == 0:
        return laplace7(16 if small else 32, seed=0)
    if k == 1:
        return multipart_aniso(12 if small else 64, seed=1)
    if k == 2:
        return var27(20 if small else 256, block=4 if small else 8, seed=2)
    if k == 3:
        if small:
            return batched(nprob=3, nrhs=4, seed=3, pmax=3, emin=4, emax=10)
        return batched(nprob=64, nrhs=4, seed=3)
    if k == 4:
        return diffusion_exp(16 if small else 128, seed=4, nfd=8 if small else 32)
    if k == 5:
        return three_point(8 if small else 160, seed=5)
    if k == 6:
        return samr(8 if small else 128, seed=6)
    if k == 7:
        return multibox(4 if small else 96, seed=7)
    raise ValueError(k)
