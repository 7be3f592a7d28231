"""SSAMG in plain numpy, FP64 (test infrastructure only; see package header).

Conventions (the readings of the paper this oracle takes):

* Grid (Section 2): part p is one box [lo, hi] (inclusive, absolute indices
  in the part's own index space), or a group of boxes held over their
  bounding box [lo, hi] with the cells outside them decoupled (diagonal 1,
  no connections).  Arrays are indexed [k, j, i]; vectors are part-major
  with i fastest.
* S (Section 2): S(c, c+o) = a_o(c) when c+o lies inside the part box, zero
  otherwise (physical boundaries are eliminated; connections across parts
  live in U).
* U (Section 2): COO entries (row, col, value) between cells of different
  parts, each tagged with direction bits: bit 2d (+d) or 2d+1 (-d) for the
  offset that leaves the part.
* Coarse points (Section 3.2, Fig. interp): cells with an even absolute index
  along the coarsening direction d*; coarse index = i / 2; coarse box along
  d* is [ceil(lo/2), floor(hi/2)].
* Interpolation sign (Eq. prolEx, printed without a minus sign): P_W =
  -(sum of the -1 plane) / (sum of the centre plane), P_E likewise, which
  gives weights in [0, 1] for M-matrices.
* Part-boundary fix (Section 3.2): a fine point whose U row carries the
  direction bit +d* (-d*), i.e. whose neighbour that way lies outside its
  part and across a coupled part boundary, gets 0 on that side and 1 on the
  other side (row sum one).
* Coarsening stop (Section 3.1): the coarsest level is the first whose total
  size is <= s_max, or level l_max - 1, or the first with every part at one
  cell.
* Relaxation weight (Section 3.4): omega_p uses W_p at level l before
  Algorithm 1 doubles it, and the d* chosen at that level.
* Coarsest level: dense Cholesky solve (default) or one relaxation sweep
  (Section 3.5, non-hybrid case).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

__all__ = [
    "Level", "Hierarchy", "Params", "level0_from_problem", "coupling_sums", "grid_spacings",
    "choose_direction", "relaxation_weight", "coarsen_box", "coarsen_plan", "interpolation",
    "prolongation_coo", "galerkin_structured", "galerkin_unstructured", "smoother_inverse",
    "matvec", "structured_matvec", "unstructured_matvec", "prolong", "restrict", "setup",
    "vcycle", "pcg", "coef_gradient", "diffusion_exp_gradient", "coarse_operator_dense",
]

Offset = Tuple[int, int, int]


# ---------------------------------------------------------------------------
# Data structures
# ---------------------------------------------------------------------------

@dataclass
class Params:
    relax: int = 0                # 0 weighted Jacobi (Eq. relax1), 1 L1-Jacobi
    relax_factor: float = 0.0     # <= 0: paper's omega_p (wJacobi) / 3/2 (L1)
    max_levels: int = 64          # l_max
    s_max: int = 0                # <= 0: number of parts
    tol: float = 1e-8
    max_iter: int = 200
    coarse_direct: int = 1        # 1: dense Cholesky, 0: one relaxation sweep
    skip: int = 0                 # the "skip" option of Section 3.4: 0 off, 1 rounds reading,
                                  # 2 literal test (see skipped_parts)
    spacings: Optional[np.ndarray] = None  # user "representative grid spacings" (n_parts x 3),
                                  # used for coarsening instead of W from the coefficients (3.1)


@dataclass
class Level:
    ndim: int
    lo: List[np.ndarray]
    hi: List[np.ndarray]
    S: List[Dict[Offset, np.ndarray]]          # per part: offset -> (nz, ny, nx)
    u_row: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    u_col: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    u_val: np.ndarray = field(default_factory=lambda: np.zeros(0))
    u_bits: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    # filled by the setup
    dstar: List[int] = field(default_factory=list)    # -1: part not coarsened
    omega: List[float] = field(default_factory=list)
    PW: List[Optional[np.ndarray]] = field(default_factory=list)
    PE: List[Optional[np.ndarray]] = field(default_factory=list)
    P: Optional[Tuple[np.ndarray, np.ndarray, np.ndarray]] = None   # COO fine->coarse
    Dinv: Optional[np.ndarray] = None

    @property
    def nparts(self):
        return len(self.lo)

    def shape(self, p):
        e = self.hi[p] - self.lo[p] + 1
        return (int(e[2]), int(e[1]), int(e[0]))

    def sizes(self):
        return [int(np.prod(self.shape(p))) for p in range(self.nparts)]

    def offsets(self):
        return np.concatenate([[0], np.cumsum(self.sizes())]).astype(np.int64)

    @property
    def n(self):
        return int(sum(self.sizes()))

    def part_view(self, v, p):
        o = self.offsets()
        return v[o[p]:o[p + 1]].reshape(self.shape(p))

    def global_index(self, p, idx_abs):
        """Global vector index of absolute cells idx_abs (m, 3) of part p."""
        loc = np.asarray(idx_abs) - self.lo[p]
        nz, ny, nx = self.shape(p)
        return self.offsets()[p] + (loc[:, 2] * ny + loc[:, 1]) * nx + loc[:, 0]

    def locate(self, g):
        """Part id and absolute (i, j, k) of global indices g."""
        o = self.offsets()
        p = np.searchsorted(o, g, side="right") - 1
        ijk = np.zeros((len(g), 3), np.int64)
        for q in np.unique(p):
            m = p == q
            nz, ny, nx = self.shape(q)
            t = g[m] - o[q]
            ijk[m, 0] = t % nx + self.lo[q][0]
            ijk[m, 1] = (t // nx) % ny + self.lo[q][1]
            ijk[m, 2] = t // (nx * ny) + self.lo[q][2]
        return p, ijk


@dataclass
class Hierarchy:
    levels: List[Level]
    params: Params
    W0: np.ndarray
    chol: Optional[np.ndarray] = None

    @property
    def L(self):
        return len(self.levels) - 1


# ---------------------------------------------------------------------------
# Small helpers (zero-filled shifts of part arrays)
# ---------------------------------------------------------------------------

def _shift(arr: np.ndarray, o: Offset) -> np.ndarray:
    """out[c] = arr[c + o] (o = (ox, oy, oz)); zero where c + o leaves the box."""
    out = np.zeros_like(arr)
    src, dst = [], []
    for ax, oo in zip((0, 1, 2), (o[2], o[1], o[0])):
        n = arr.shape[ax]
        if abs(oo) >= n:
            return out
        dst.append(slice(max(0, -oo), n - max(0, oo)))
        src.append(slice(max(0, oo), n - max(0, -oo)))
    out[tuple(dst)] = arr[tuple(src)]
    return out


def _inside_mask(shape, o: Offset) -> np.ndarray:
    """True where c + o is inside a box of the given (nz, ny, nx) shape."""
    return _shift(np.ones(shape), o) > 0


def _ceil_half(v):
    return -((-v) // 2)


def _unit(d, s=1):
    o = [0, 0, 0]
    o[d] = s
    return tuple(o)


# ---------------------------------------------------------------------------
# Level 0 from a problem description (Section 2: A = S + U)
# ---------------------------------------------------------------------------

def part_active(prob, p, shp) -> np.ndarray:
    """Cells of part p's bounding box that belong to the part (Section 2: a
    part is a group of boxes); all of them for a one-box part."""
    boxes = prob.part_boxes[p] if getattr(prob, "part_boxes", None) else None
    m = np.zeros(shp, bool)
    if boxes is None:
        m[...] = True
        return m
    lo = prob.boxes[p][0]
    zz, yy, xx = np.meshgrid(*(np.arange(n) + l for n, l in zip(shp, (lo[2], lo[1], lo[0]))),
                             indexing="ij")
    for blo, bhi in boxes:
        m |= ((xx >= blo[0]) & (xx <= bhi[0]) & (yy >= blo[1]) & (yy <= bhi[1]) &
              (zz >= blo[2]) & (zz <= bhi[2]))
    return m


def level0_from_problem(prob) -> Level:
    """S with out-of-box connections dropped, U with duplicates summed.

    A part of several boxes is held over its bounding box: connections from
    or to a cell outside its boxes are dropped and such a cell is a decoupled
    unknown (diagonal 1), as the paper's ghost unknowns (Section 4, test case
    4); stencil connections between the part's boxes stay (interpolation
    within a part crosses its box faces)."""
    lo = [np.array(b[0], np.int64) for b in prob.boxes]
    hi = [np.array(b[1], np.int64) for b in prob.boxes]
    S = []
    for p in range(prob.nparts):
        e = hi[p] - lo[p] + 1
        shp = (int(e[2]), int(e[1]), int(e[0]))
        act = part_active(prob, p, shp)
        sp = {}
        for ei, o in enumerate(prob.offsets):
            o = tuple(int(v) for v in o)
            c = prob.coef[p][ei]
            arr = np.full(shp, float(c)) if np.isscalar(c) else np.array(c, np.float64).reshape(shp)
            arr = np.where(_inside_mask(shp, o), arr, 0.0)
            if not act.all():
                if o == (0, 0, 0):
                    arr = np.where(act, arr, 1.0)
                else:
                    arr = np.where(act & _shift(act, o), arr, 0.0)
            sp[o] = sp.get(o, 0.0) + arr
        S.append(sp)
    lev = Level(prob.ndim, lo, hi, S)
    if prob.nnz_u:
        rows = np.zeros(prob.nnz_u, np.int64)
        cols = np.zeros(prob.nnz_u, np.int64)
        for p in range(prob.nparts):
            m = prob.u_part == p
            rows[m] = lev.global_index(p, prob.u_idx[m])
            mq = prob.u_nbor_part == p
            cols[mq] = lev.global_index(p, prob.u_nbor_idx[mq])
        bits = np.zeros(prob.nnz_u, np.int64)
        for d in range(3):
            bits |= np.where(prob.u_dir[:, d] > 0, 1 << (2 * d), 0)
            bits |= np.where(prob.u_dir[:, d] < 0, 1 << (2 * d + 1), 0)
        lev.u_row, lev.u_col, lev.u_val, lev.u_bits = _coo_sum(rows, cols, prob.u_val, bits, lev.n)
    return lev


def _coo_sum(rows, cols, vals, bits, n):
    """Sum duplicate (row, col) pairs, OR their direction bits; sort by row, col."""
    if len(rows) == 0:
        z = np.zeros(0, np.int64)
        return z, z.copy(), np.zeros(0), z.copy()
    key = rows.astype(np.int64) * n + cols.astype(np.int64)
    uk, inv = np.unique(key, return_inverse=True)
    v = np.zeros(len(uk))
    np.add.at(v, inv, vals)
    bb = np.zeros(len(uk), np.int64)
    np.bitwise_or.at(bb, inv, bits.astype(np.int64))
    return uk // n, uk % n, v, bb


# ---------------------------------------------------------------------------
# Operator application (Section 2 and Eq. relax0)
# ---------------------------------------------------------------------------

def structured_matvec(lev: Level, x: np.ndarray) -> np.ndarray:
    """y = S x, part by part, one stencil entry at a time."""
    y = np.zeros(lev.n)
    for p in range(lev.nparts):
        xp = lev.part_view(x, p)
        yp = lev.part_view(y, p)
        for o, a in lev.S[p].items():
            yp += a * _shift(xp, o)
    return y


def unstructured_matvec(lev: Level, x: np.ndarray) -> np.ndarray:
    """y = U x from the COO entries."""
    y = np.zeros(lev.n)
    if len(lev.u_val):
        np.add.at(y, lev.u_row, lev.u_val * x[lev.u_col])
    return y


def matvec(lev: Level, x: np.ndarray) -> np.ndarray:
    return structured_matvec(lev, x) + unstructured_matvec(lev, x)


# ---------------------------------------------------------------------------
# Coarsening (Section 3.1)
# ---------------------------------------------------------------------------

def coupling_sums(lev: Level) -> np.ndarray:
    """c[p, d]: over all cells of part p, the negated sum of the stencil
    coefficients whose offset moves along d (Section 3.1, equation for c_1),
    each cell's contribution sign-adjusted so that its diagonal is positive."""
    c = np.zeros((lev.nparts, 3))
    for p in range(lev.nparts):
        diag = lev.S[p].get((0, 0, 0))
        sgn = np.ones(lev.shape(p)) if diag is None else np.where(diag < 0, -1.0, 1.0)
        for d in range(3):
            acc = np.zeros(lev.shape(p))
            for o, a in lev.S[p].items():
                if o[d] != 0:
                    acc -= a
            c[p, d] = float(np.sum(sgn * acc))
    return c


def grid_spacings(c: np.ndarray, ndim: int) -> np.ndarray:
    """W[p, d] = sqrt(max_i c_i / c_d) (Section 3.1); +inf where c_d <= 0 or
    d >= ndim."""
    W = np.full(c.shape, np.inf)
    for p in range(c.shape[0]):
        cmax = max(c[p, :ndim])
        for d in range(ndim):
            if c[p, d] > 0 and cmax > 0:
                W[p, d] = math.sqrt(cmax / c[p, d])
    return W


def user_spacings(W, prob) -> np.ndarray:
    """Representative grid spacings given by the user (Section 3.1: an option
    kept from PFMG, used only for coarsening): n_parts x 3, positive or +inf;
    dimensions >= ndim are +inf."""
    W = np.array(W, dtype=float).reshape(prob.nparts, 3)
    if np.any(np.isnan(W)) or np.any(W <= 0):
        raise ValueError("spacings must be positive (or +inf)")
    W[:, prob.ndim:] = np.inf
    return W


def choose_direction(Wp: np.ndarray, extent: np.ndarray, ndim: int) -> int:
    """argmin_d W_pd over dimensions the box can still be halved in; ties go
    to the smallest index (Section 3.1 footnote).  With no such dimension,
    the argmin over all dimensions."""
    cand = [d for d in range(ndim) if extent[d] > 1]
    if not cand:
        cand = list(range(ndim))
    best = cand[0]
    for d in cand[1:]:
        if Wp[d] < Wp[best]:
            best = d
    return best


def relaxation_weight(Wp: np.ndarray, dstar: int, ndim: int) -> float:
    """omega_p = 2 / (3 - beta_p/alpha_p) (Eqs. relax1 and alpha-beta)."""
    inv = [0.0 if not np.isfinite(Wp[d]) else 1.0 / (Wp[d] * Wp[d]) for d in range(ndim)]
    alpha = sum(inv)
    beta = alpha - inv[dstar]
    if alpha <= 0.0:
        return 1.0
    return 2.0 / (3.0 - beta / alpha)


def coarsen_box(lo, hi, d):
    """Halve a box along d: coarse cells are the even indices, I = i/2."""
    lo2, hi2 = lo.copy(), hi.copy()
    lo2[d] = _ceil_half(lo[d])
    hi2[d] = hi[d] // 2
    return lo2, hi2


def coarsen_plan(W0, lo0, hi0, ndim, s_max, l_max):
    """Algorithm 1: per level, per part, d* and the coarsened bounding box.

    Returns (boxes per level, dstar per level, omega per level).  dstar = -1
    marks a part that is not coarsened at that level (volume one) and every
    part of the coarsest level.
    """
    W = W0.copy()
    boxes = [(list(lo0), list(hi0))]
    dstars, omegas = [], []
    nparts = len(lo0)
    while True:
        lo, hi = boxes[-1]
        vol = [int(np.prod(hi[p] - lo[p] + 1)) for p in range(nparts)]
        total = sum(vol)
        if total <= s_max or len(boxes) >= l_max or all(v <= 1 for v in vol):
            ds = [choose_direction(W[p], hi[p] - lo[p] + 1, ndim) for p in range(nparts)]
            omegas.append([relaxation_weight(W[p], ds[p], ndim) for p in range(nparts)])
            dstars.append([-1] * nparts)
            break
        nlo, nhi, ds, om = [], [], [], []
        for p in range(nparts):
            ext = hi[p] - lo[p] + 1
            d = choose_direction(W[p], ext, ndim)
            om.append(relaxation_weight(W[p], d, ndim))
            if vol[p] > 1:
                a, b = coarsen_box(lo[p], hi[p], d)
                W[p, d] *= 2.0
                ds.append(d)
            else:
                a, b = lo[p].copy(), hi[p].copy()
                ds.append(-1)
            nlo.append(a)
            nhi.append(b)
        dstars.append(ds)
        omegas.append(om)
        boxes.append((nlo, nhi))
    return boxes, dstars, omegas


# ---------------------------------------------------------------------------
# Interpolation (Section 3.2, Eq. prolEx)
# ---------------------------------------------------------------------------

def _face_bits(lev: Level, p: int) -> np.ndarray:
    """OR of the U direction bits of each cell's row (shape of part p)."""
    bits = np.zeros(lev.n, np.int64)
    if len(lev.u_row):
        np.bitwise_or.at(bits, lev.u_row, lev.u_bits)
    return lev.part_view(bits, p)


def interpolation(lev: Level, p: int, d: int):
    """Two-point weights (PW, PE) of part p along d, on the fine grid.

    For a fine point f (odd absolute index along d):
      PW = -(sum of S entries with offset_d = -1) / (sum with offset_d = 0)
      PE = -(sum of S entries with offset_d = +1) / (same denominator)
    Entries leaving the box are already zero in S.  A denominator that is
    (numerically) zero or whose sign differs from the diagonal gives zero
    weights.  Part-boundary fix: across a coupled face the weight is 0 and the
    opposite weight is 1.  Coarse points carry (0, 0) here; their weight 1 is
    implied.
    """
    shp = lev.shape(p)
    S = lev.S[p]
    num_w = np.zeros(shp)
    num_e = np.zeros(shp)
    den = np.zeros(shp)
    for o, a in S.items():
        if o[d] == -1:
            num_w += a
        elif o[d] == 1:
            num_e += a
        else:
            den += a
    diag = S.get((0, 0, 0), np.zeros(shp))
    ok = (np.abs(den) > 1e-300) & (np.sign(den) == np.sign(diag))
    safe = np.where(ok, den, 1.0)
    PW = np.where(ok, -num_w / safe, 0.0)
    PE = np.where(ok, -num_e / safe, 0.0)
    ax = 2 - d
    idx = np.arange(shp[ax]) + lev.lo[p][d]
    bshape = [1, 1, 1]
    bshape[ax] = shp[ax]
    fine = np.broadcast_to((idx % 2 == 1).reshape(bshape), shp)
    bits = _face_bits(lev, p)
    # a row's bit +d (-d) says that it leaves its part through +d (-d): on
    # the box face for a one-box part, also beside a hole for a part of
    # several boxes
    cross_e = fine & ((bits >> (2 * d)) & 1).astype(bool)
    cross_w = fine & ((bits >> (2 * d + 1)) & 1).astype(bool)
    PE = np.where(cross_e, 0.0, PE)
    PW = np.where(cross_e, 1.0, PW)
    PW = np.where(cross_w, 0.0, PW)
    PE = np.where(cross_w, 1.0, PE)
    PW = np.where(fine, PW, 0.0)
    PE = np.where(fine, PE, 0.0)
    return PW, PE


def _prolongation_columns(fine: Level, coarse: Level, p: int, g_abs: np.ndarray):
    """For absolute fine cells g_abs (m, 3) of part p: up to two (coarse
    global index, weight) pairs of P's row; index -1 marks an absent entry."""
    m = len(g_abs)
    cols = np.full((m, 2), -1, np.int64)
    wts = np.zeros((m, 2))
    d = fine.dstar[p]
    if d < 0:
        cols[:, 0] = coarse.global_index(p, g_abs)
        wts[:, 0] = 1.0
        return cols, wts
    gl = fine.global_index(p, g_abs)
    lo_c, hi_c = coarse.lo[p][d], coarse.hi[p][d]
    gd = g_abs[:, d]
    even = gd % 2 == 0
    J = g_abs.copy()
    J[:, d] = gd // 2
    if even.any():
        cols[even, 0] = coarse.global_index(p, J[even])
        wts[even, 0] = 1.0
    odd = ~even
    PWf = fine.PW[p].reshape(-1)
    PEf = fine.PE[p].reshape(-1)
    loc = gl - fine.offsets()[p]
    Jw = g_abs.copy()
    Jw[:, d] = (gd - 1) // 2
    Je = g_abs.copy()
    Je[:, d] = (gd + 1) // 2
    mw = odd & (Jw[:, d] >= lo_c)
    me = odd & (Je[:, d] <= hi_c)
    if mw.any():
        cols[mw, 0] = coarse.global_index(p, Jw[mw])
        wts[mw, 0] = PWf[loc[mw]]
    if me.any():
        cols[me, 1] = coarse.global_index(p, Je[me])
        wts[me, 1] = PEf[loc[me]]
    return cols, wts


def prolongation_coo(fine: Level, coarse: Level):
    """Explicit P (rows = fine global, cols = coarse global, values)."""
    R, C, V = [], [], []
    for p in range(fine.nparts):
        nz, ny, nx = fine.shape(p)
        kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        g_abs = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1) + fine.lo[p]
        cols, wts = _prolongation_columns(fine, coarse, p, g_abs)
        rows = fine.global_index(p, g_abs)
        for s in range(2):
            m = cols[:, s] >= 0
            R.append(rows[m])
            C.append(cols[m, s])
            V.append(wts[m, s])
    return np.concatenate(R), np.concatenate(C), np.concatenate(V)


def prolong(lev: Level, ec: np.ndarray) -> np.ndarray:
    """P e_c."""
    r, c, v = lev.P
    return np.bincount(r, weights=v * ec[c], minlength=lev.n)


def restrict(lev: Level, r_f: np.ndarray, n_coarse: int) -> np.ndarray:
    """R r = P^T r (Section 3.2: Galerkin restriction)."""
    r, c, v = lev.P
    return np.bincount(c, weights=v * r_f[r], minlength=n_coarse)


# ---------------------------------------------------------------------------
# Coarse operator (Section 3.3, Eq. galerkin)
# ---------------------------------------------------------------------------

def galerkin_structured(fine: Level, coarse: Level, p: int) -> Dict[Offset, np.ndarray]:
    """P^T S P for part p as coarse stencils.

    For coarse cell I with fine anchor F = 2I along d* and each a in
    {-1, 0, 1}: f = F + a e_d has weight P(f, I) = 1 (a = 0), PE(f) (a = -1)
    or PW(f) (a = +1).  For each fine entry o at f, g = f + o: if g is a
    coarse point it maps to J = g/2 with weight 1; otherwise to its west and
    east coarse neighbours with PW(g) and PE(g).  The product
    P(f, I) a_o(f) P(g, J) accumulates into the coarse entry J - I.
    """
    d = fine.dstar[p]
    S = fine.S[p]
    if d < 0:
        return {o: a.copy() for o, a in S.items()}
    shp_c = coarse.shape(p)
    ax = 2 - d
    # anchors: fine local index of each coarse point along d
    anchors = 2 * (np.arange(shp_c[ax]) + coarse.lo[p][d]) - fine.lo[p][d]

    def at_anchor(arr):
        return np.take(arr, anchors, axis=ax)

    ones = np.ones(fine.shape(p))
    w_to_I = {0: ones, -1: fine.PE[p], 1: fine.PW[p]}
    out: Dict[Offset, np.ndarray] = {}
    for a in (-1, 0, 1):
        sa = _unit(d, a)
        w1 = at_anchor(_shift(w_to_I[a], sa))
        for o, coef in S.items():
            c1 = at_anchor(_shift(coef, sa)) * w1
            go = tuple(sa[i] + o[i] for i in range(3))       # g - F
            t = a + o[d]
            if t % 2 == 0:
                targets = [(t // 2, None)]
            else:
                targets = [((t - 1) // 2, fine.PW[p]), ((t + 1) // 2, fine.PE[p])]
            for jd, warr in targets:
                w2 = 1.0 if warr is None else at_anchor(_shift(warr, go))
                oc = list(o)
                oc[d] = jd
                oc = tuple(oc)
                out[oc] = out.get(oc, 0.0) + c1 * w2
    return out


def galerkin_unstructured(fine: Level, coarse: Level):
    """P^T U P: each U entry (f, g, v) spreads to P(f, I) v P(g, J)."""
    if len(fine.u_row) == 0:
        z = np.zeros(0, np.int64)
        return z, z.copy(), np.zeros(0), z.copy()
    pr, ijr = fine.locate(fine.u_row)
    pc, ijc = fine.locate(fine.u_col)
    m = len(fine.u_row)
    Ic = np.full((m, 2), -1, np.int64)
    Iw = np.zeros((m, 2))
    Jc = np.full((m, 2), -1, np.int64)
    Jw = np.zeros((m, 2))
    for q in range(fine.nparts):
        mr = pr == q
        if mr.any():
            Ic[mr], Iw[mr] = _prolongation_columns(fine, coarse, q, ijr[mr])
        mc = pc == q
        if mc.any():
            Jc[mc], Jw[mc] = _prolongation_columns(fine, coarse, q, ijc[mc])
    R, C, V, B = [], [], [], []
    for s1 in range(2):
        for s2 in range(2):
            ok = (Ic[:, s1] >= 0) & (Jc[:, s2] >= 0)
            R.append(Ic[ok, s1])
            C.append(Jc[ok, s2])
            V.append(Iw[ok, s1] * fine.u_val[ok] * Jw[ok, s2])
            B.append(fine.u_bits[ok])
    return _coo_sum(np.concatenate(R), np.concatenate(C), np.concatenate(V),
                    np.concatenate(B), coarse.n)


# ---------------------------------------------------------------------------
# Relaxation (Section 3.4)
# ---------------------------------------------------------------------------

def skipped_parts(dstars, ndim: int, l: int, mode: int = 1) -> List[bool]:
    """The "skip" option of Section 3.4: which parts do no relaxation at level l.

    The paper states the test d*_l = d*_{l - n_d} and says that the option
    mimics full coarsening; Section 4 (test case 2) adds that a part coarsened
    along one direction for its first levels has relaxation skipped only on
    later levels.  Applied alone at every level, the test would stop an
    isotropic part from relaxing anywhere below level n_d, which is not full
    coarsening, and would skip level n_d of a part still coarsening along its
    strong direction.

    mode 1 (the reading taken): per part, the levels form rounds as full
    coarsening would: a round starts at level 0 and at every level whose d*
    already occurs in the current round, so a round holds distinct
    directions (at most n_d).  A part with d*_l = d*_{l - n_d} throughout
    (isotropic: x, y, z, x, ...) gets rounds [0, n_d), [n_d, 2 n_d), ...;
    relaxation stays on the first level of each round and is off on the
    others, i.e. on levels 0, n_d, 2 n_d, ..., the grids full coarsening
    visits.  A repeated direction (the strong direction of an anisotropic
    part) starts a new round at each repetition, so those levels keep
    relaxing.  A level where the part is not coarsened (d* = -1: one cell, or
    the coarsest level) relaxes and ends the round.

    mode 2: the test read literally: skip level l >= n_d when d*_l >= 0 and
    d*_l = d*_{l - n_d}.
    """
    nparts = len(dstars[l])
    if mode == 2:
        if l < ndim:
            return [False] * nparts
        return [dstars[l][p] >= 0 and dstars[l][p] == dstars[l - ndim][p] for p in range(nparts)]
    out = []
    for p in range(nparts):
        seen = set()
        skip = False
        for k in range(l + 1):
            d = dstars[k][p]
            if d < 0 or d in seen:
                seen = set() if d < 0 else {d}
                skip = False
            elif not seen:
                seen = {d}
                skip = False
            else:
                seen.add(d)
                skip = True
        out.append(skip)
    return out


def smoother_inverse(lev: Level, params: Params) -> np.ndarray:
    """The diagonal of omega M^-1 in Eq. relax0.

    Weighted Jacobi: omega_p / A_ii (omega_p from Eq. relax1 unless the user
    gives a factor).  L1 Jacobi: factor / sum_j |A_ij| over S and U, factor
    3/2 by default (the paper's SSAMG-base setting).
    """
    out = np.zeros(lev.n)
    l1u = np.zeros(lev.n)
    if params.relax == 1 and len(lev.u_val):
        np.add.at(l1u, lev.u_row, np.abs(lev.u_val))
    skip = getattr(lev, "skip", None)
    for p in range(lev.nparts):
        dv = lev.part_view(out, p)
        if skip is not None and skip[p]:
            continue  # relaxation turned off: omega M^-1 = 0 (x stays 0 / unchanged)
        if params.relax == 0:
            w = params.relax_factor if params.relax_factor > 0 else lev.omega[p]
            dv[...] = w / lev.S[p][(0, 0, 0)]
        else:
            w = params.relax_factor if params.relax_factor > 0 else 1.5
            s = lev.part_view(l1u, p).copy()
            for a in lev.S[p].values():
                s += np.abs(a)
            dv[...] = w / s
    return out


# ---------------------------------------------------------------------------
# Setup
# ---------------------------------------------------------------------------

def coarse_operator_dense(lev: Level) -> np.ndarray:
    """The coarsest operator as a dense matrix (columns = A e_j)."""
    n = lev.n
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = matvec(lev, e)
    return A


def setup(prob, params: Params = Params()) -> Hierarchy:
    lev0 = level0_from_problem(prob)
    c = coupling_sums(lev0)
    W0 = grid_spacings(c, prob.ndim) if params.spacings is None else user_spacings(params.spacings, prob)
    s_max = params.s_max if params.s_max > 0 else prob.nparts
    boxes, dstars, omegas = coarsen_plan(W0, lev0.lo, lev0.hi, prob.ndim, s_max, params.max_levels)
    levels = [lev0]
    for l in range(len(boxes)):
        fine = levels[l]
        fine.dstar = dstars[l]
        fine.omega = omegas[l]
        if l == len(boxes) - 1:
            break
        nlo, nhi = boxes[l + 1]
        coarse = Level(prob.ndim, [np.array(v) for v in nlo], [np.array(v) for v in nhi],
                       [None] * fine.nparts)
        fine.PW, fine.PE = [None] * fine.nparts, [None] * fine.nparts
        for p in range(fine.nparts):
            if fine.dstar[p] >= 0:
                fine.PW[p], fine.PE[p] = interpolation(fine, p, fine.dstar[p])
        fine.P = prolongation_coo(fine, coarse)
        for p in range(fine.nparts):
            coarse.S[p] = galerkin_structured(fine, coarse, p)
        coarse.u_row, coarse.u_col, coarse.u_val, coarse.u_bits = galerkin_unstructured(fine, coarse)
        levels.append(coarse)
    for l, lev in enumerate(levels):
        lev.skip = (skipped_parts(dstars, prob.ndim, l, params.skip) if params.skip and l < len(dstars)
                    else [False] * lev.nparts)
        lev.Dinv = smoother_inverse(lev, params)
    h = Hierarchy(levels, params, W0)
    if params.coarse_direct:
        h.chol = np.linalg.cholesky(coarse_operator_dense(levels[-1]))
    return h


# ---------------------------------------------------------------------------
# V(1,1) cycle and PCG (Sections 3.4, 3.5 and 4)
# ---------------------------------------------------------------------------

def _coarse_solve(h: Hierarchy, b: np.ndarray) -> np.ndarray:
    if h.chol is not None:
        y = np.linalg.solve(h.chol, b)
        return np.linalg.solve(h.chol.T, y)
    return h.levels[-1].Dinv * b


def vcycle(h: Hierarchy, b: np.ndarray, l: int = 0) -> np.ndarray:
    """One V(1,1) cycle from a zero initial guess: pre-relax, restrict the
    residual, recurse, prolong-correct, post-relax."""
    if l == h.L:
        return _coarse_solve(h, b)
    lev = h.levels[l]
    x = lev.Dinv * b
    r = b - matvec(lev, x)
    bc = restrict(lev, r, h.levels[l + 1].n)
    x = x + prolong(lev, vcycle(h, bc, l + 1))
    x = x + lev.Dinv * (b - matvec(lev, x))
    return x


@dataclass
class PCGResult:
    x: np.ndarray
    iterations: int
    converged: bool
    rel_res: float
    true_rel_res: float
    history: List[float]


def pcg(h: Hierarchy, b: np.ndarray, tol: Optional[float] = None, max_iter: Optional[int] = None,
        x0: Optional[np.ndarray] = None) -> PCGResult:
    """Conjugate gradients preconditioned by one V-cycle per iteration.

    Stops when ||r_k||_2 <= tol ||b||_2 on the recursively updated residual.
    """
    tol = h.params.tol if tol is None else tol
    max_iter = h.params.max_iter if max_iter is None else max_iter
    A = h.levels[0]
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - matvec(A, x)
    bn = float(np.sqrt(b @ b))
    hist = [float(np.sqrt(r @ r)) / bn if bn > 0 else 0.0]
    if bn == 0.0 or hist[0] <= tol:
        return PCGResult(x, 0, True, hist[0], hist[0], hist)
    z = vcycle(h, r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    conv = False
    while it < max_iter:
        it += 1
        q = matvec(A, p)
        pq = float(p @ q)
        if not (pq > 0.0) or not np.isfinite(pq):
            raise FloatingPointError("PCG breakdown: p.Ap <= 0")
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        rn = float(np.sqrt(r @ r)) / bn
        hist.append(rn)
        if rn <= tol:
            conv = True
            break
        z = vcycle(h, r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    tr = b - matvec(A, x)
    return PCGResult(x, it, conv, hist[-1], float(np.sqrt(tr @ tr)) / bn, hist)


# ---------------------------------------------------------------------------
# Differentiation (adjoint of the linear solve; not part of the paper)
# ---------------------------------------------------------------------------

def coef_gradient(lev: Level, lam: np.ndarray, x: np.ndarray):
    """dL/da_o(c) = -lambda_c x_{c+o} for every stencil entry inside the box
    (from dL/dA = -lambda x^T with A lambda = dL/dx)."""
    out = []
    for p in range(lev.nparts):
        lp = lev.part_view(lam, p)
        xp = lev.part_view(x, p)
        out.append({o: np.where(_inside_mask(lev.shape(p), o), -lp * _shift(xp, o), 0.0)
                    for o in lev.S[p]})
    return out


def diffusion_exp_gradient(g: np.ndarray, lam: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dL/dg for the 7-point harmonic-mean diffusion operator with kappa = exp(g).

    For an interior face (c, n) with t = 2 k_c k_n / (k_c + k_n):
    dL/dt = -(lam_c - lam_n)(x_c - x_n) and dt/dk_c = 2 k_n^2 / (k_c + k_n)^2.
    A Dirichlet face adds k_c to A_cc, so dL/dk_c += -lam_c x_c.
    dL/dg_c = k_c dL/dk_c.
    """
    k = np.exp(g)
    lam = lam.reshape(g.shape)
    x = x.reshape(g.shape)
    dk = np.zeros_like(g)
    for d in range(3):
        for s in (-1, 1):
            o = _unit(d, s)
            inside = _inside_mask(g.shape, o)
            kn = _shift(k, o)
            ln = _shift(lam, o)
            xn = _shift(x, o)
            dt = np.where(inside, 2.0 * kn * kn / np.where(inside, (k + kn) ** 2, 1.0), 0.0)
            dk += np.where(inside, -dt * (lam - ln) * (x - xn), -lam * x)
    return k * dk
