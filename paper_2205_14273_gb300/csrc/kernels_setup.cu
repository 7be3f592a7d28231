// Setup kernels: coupling sums (Section 3.1), interpolation (Section 3.2,
// Eq. prolEx), Galerkin coarse operators (Section 3.3, Eq. galerkin),
// relaxation diagonals (Section 3.4) and the coarsest-level factorisation.
#include <climits>

#include "kernels_common.cuh"

namespace {

constexpr int NT = SSAMG_BLOCK;

// P's row as column and weight arrays J[0..m), w[0..m) (the first the west or
// only column); returns m.  Unused slots hold -1 and 0.
template <class T>
__device__ __forceinline__ int p_row_arrays(const DPart& p, const T* __restrict__ Pw,
                                            const T* __restrict__ Pe, int i, int j, int k, int* J,
                                            T* w) {
  const PRow<T> r = p_row(p, Pw, Pe, i, j, k);
  J[0] = r.j0;
  w[0] = r.w0;
  J[1] = r.j1;
  w[1] = r.w1;
  return (r.j0 >= 0) + (r.j1 >= 0);
}

// ---------------------------------------------------------------------------
// K1: per part, c_d = sum over cells of sign(A_C) * (-sum of entries moving
// along d) (Section 3.1).  Block partials, then one block per part sums them
// in a fixed order.
// ---------------------------------------------------------------------------
// Constant entries (one value over the part) contribute -a_e times the
// number of the block's cells whose neighbour c + o_e is in the box, each
// counted with the cell's sign: exact integers (a warp sum per step, kept by
// the warp's lane 0), multiplied once per block; per-cell entries are summed
// in FP64 cell by cell.  The diagonal's sign is read from its bits (negative,
// nonzero, not NaN: the same decision as diag < 0).
__global__ void __launch_bounds__(NT) k_wsum(LevelView<double> L, double* __restrict__ partial) {
  __shared__ DPart sp;
  __shared__ double sh[NT];
  __shared__ int shc[NT / 32][SSAMG_MAXE];
  int p = block_part(L.blk, L.parts, L.np, sp);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0)
    for (int e = 0; e < SSAMG_MAXE; ++e) shc[w][e] = 0;
  __syncthreads();
  int de = -1;  // the diagonal entry (offset 0, 0, 0)
  bool anyvar = false;
  for (int e = 0; e < sp.nent; ++e) {
    if (sp.o[e][0] == 0 && sp.o[e][1] == 0 && sp.o[e][2] == 0)
      de = e;
    else if (sp.coef[e] >= 0)
      anyvar = true;
  }
  double s0 = 0, s1 = 0, s2 = 0;
  const int base = ((int)blockIdx.x - sp.blk0) * sp.cpt * SSAMG_BLOCK + (int)threadIdx.x;
#pragma unroll 1
  for (int m = 0; m < sp.cpt; ++m) {
    const int c = base + m * SSAMG_BLOCK;
    if (c - lane >= sp.ncell) break;  // the warp's first cell: a warp-uniform exit
    const bool valid = c < sp.ncell;
    int i = 0, j = 0, k = 0;
    bool neg = false;
    if (valid) {
      cell_coords(sp, c, i, j, k);
      if (de >= 0) {
        const long long bits = __double_as_longlong(coef_at(sp, L.coef, de, c));
        const long long mag = bits & 0x7fffffffffffffffll;
        neg = bits < 0 && mag != 0 && mag <= 0x7ff0000000000000ll;
      }
    }
    double t0 = 0, t1 = 0, t2 = 0;
#pragma unroll 1
    for (int e = 0; e < sp.nent; ++e) {
      if (e == de) continue;
      const bool ok = valid && inside(sp, i + sp.o[e][0], j + sp.o[e][1], k + sp.o[e][2]);
      if (sp.coef[e] >= 0) {
        if (ok) {
          const double a = L.coef[sp.coef[e] + c];
          if (sp.o[e][0]) t0 -= a;
          if (sp.o[e][1]) t1 -= a;
          if (sp.o[e][2]) t2 -= a;
        }
      } else {
        const int v = __reduce_add_sync(0xffffffffu, ok ? (neg ? -1 : 1) : 0);
        if (lane == 0) shc[w][e] += v;
      }
    }
    if (anyvar && valid) {
      const double sg = neg ? -1.0 : 1.0;
      s0 += sg * t0;
      s1 += sg * t1;
      s2 += sg * t2;
    }
  }
  double r0 = block_sum<NT>(s0, sh);
  double r1 = block_sum<NT>(s1, sh);
  double r2 = block_sum<NT>(s2, sh);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int e = 0; e < sp.nent; ++e) {
      if (e == de || sp.coef[e] >= 0) continue;
      long long n = 0;
      for (int q = 0; q < NT / 32; ++q) n += shc[q][e];
      const double a = sp.cval[e] * (double)n;
      if (sp.o[e][0]) r0 -= a;
      if (sp.o[e][1]) r1 -= a;
      if (sp.o[e][2]) r2 -= a;
    }
    partial[3 * blockIdx.x + 0] = r0;
    partial[3 * blockIdx.x + 1] = r1;
    partial[3 * blockIdx.x + 2] = r2;
  }
}

__global__ void __launch_bounds__(NT) k_wfinal(const int* __restrict__ blk,
                                               const double* __restrict__ partial,
                                               double* __restrict__ c) {
  __shared__ double sh[NT];
  int p = blockIdx.x;
  int b0 = blk[p], b1 = blk[p + 1];
  for (int d = 0; d < 3; ++d) {
    double s = 0;
    for (int b = b0 + threadIdx.x; b < b1; b += NT) s += partial[3 * b + d];
    double r = block_sum<NT>(s, sh);
    if (threadIdx.x == 0) c[3 * p + d] = r;
  }
}

// ---------------------------------------------------------------------------
// K2: two-point interpolation weights per fine point (Eq. prolEx, sign
// reading P = -(plane sum)/(centre-plane sum)), with the part-boundary fix.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_interp(LevelView<double> L, double* __restrict__ Pw,
                                               double* __restrict__ Pe, float* __restrict__ Pw32,
                                               float* __restrict__ Pe32) {
  __shared__ DPart sp;
  int p = block_part(L.fblk, L.parts, L.np, sp);
  __syncthreads();
  TILE_LOOP_FINE(F, sp) {
    const int d = sp.dstar;
    int fc[3];
    {
      unsigned q = fdiv((unsigned)F, sp.fdx);
      fc[0] = F - (int)q * sp.nf[0];
      fc[2] = (int)fdiv((unsigned)F, sp.fdxy);
      fc[1] = (int)q - fc[2] * sp.nf[1];
    }
    fc[d] = 2 * fc[d] + 1 - sp.par;  // the fine cell
    const int i = fc[0], j = fc[1], k = fc[2];
    const int c = (k * sp.n[1] + j) * sp.n[0] + i;
    double nw = 0, ne = 0, den = 0, diag = 0;
    // entries in batches of IB with predicated loads (in flight together),
    // summed in entry order as before
    constexpr int IB = 9;
    for (int e0 = 0; e0 < sp.nent; e0 += IB) {
      double av[IB];
#pragma unroll
      for (int q = 0; q < IB; ++q) {
        const int e = e0 + q;
        const bool ok =
            e < sp.nent && inside(sp, i + sp.o[e][0], j + sp.o[e][1], k + sp.o[e][2]);
        av[q] = ok ? coef_at(sp, L.coef, e, c) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < IB; ++q) {
        const int e = e0 + q;
        if (e >= sp.nent) break;
        if (!inside(sp, i + sp.o[e][0], j + sp.o[e][1], k + sp.o[e][2])) continue;
        const double a = av[q];
        const int od = sp.o[e][d];
        if (od < 0) nw += a;
        else if (od > 0) ne += a;
        else den += a;
        if (sp.o[e][0] == 0 && sp.o[e][1] == 0 && sp.o[e][2] == 0) diag += a;
      }
    }
    double pw = 0, pe = 0;
    bool ok = fabs(den) > 1e-300 && ((den > 0) == (diag > 0)) && diag != 0.0;
    if (ok) {
      const double rd = 1.0 / den;  // one division for both weights
      pw = -nw * rd;
      pe = -ne * rd;
    }
    // part-boundary fix: a row's bit +d* (-d*) says that it leaves its part
    // that way (on the box face; beside a hole too when rows lie inside the
    // box, has_u = 2)
    if (sp.has_u > 1 || (sp.has_u && (fc[d] == 0 || fc[d] == sp.n[d] - 1))) {
      int r = L.u_map[sp.off + c];
      if (r >= 0) {
        unsigned bits = 0;
        for (int q = L.u_ptr[r]; q < L.u_ptr[r + 1]; ++q) bits |= L.u_bits[q];
        if ((bits >> (2 * d)) & 1u) { pw = 1.0; pe = 0.0; }
        if ((bits >> (2 * d + 1)) & 1u) { pw = 0.0; pe = 1.0; }
      }
    }
    Pw[sp.poff + F] = pw;
    Pe[sp.poff + F] = pe;
    if (Pw32) {
      Pw32[sp.poff + F] = (float)pw;
      Pe32[sp.poff + F] = (float)pe;
    }
  }
}

// ---------------------------------------------------------------------------
// K3, all levels: P^T S P with a thread per (coarse cell, off-d* offset
// group).  The coarse entries O = (u, v off d*; c along d*), c in {-1,0,1},
// of one group come only from the fine entries with the same offsets off d*
// (o_d in {-1,0,1}) at the coarse cell's three fine points f = F + a e_d
// (F its anchor 2I along d*): the product w_a s_o(f) goes to c = t/2 when
// t = a + o_d is even (g = f + o is a coarse point) and to (t-1)/2 and
// (t+1)/2 with PW(g), PE(g) when t is odd.  a and o_d are compile-time, so
// the group's three sums stay in registers; each sum runs in the order
// (a, o_d) ascending.  Each fine coefficient is read once per coarse cell.
// Block b takes group b % 9 of coarse tile b / 9.
// ---------------------------------------------------------------------------
// D: the coarsening direction of the part (-1: not coarsened, P = I), a
// template argument so that the coordinate arrays stay in registers.
template <int D>
__device__ __forceinline__ void rap_group_tile(const LevelView<double>& F, const DPart& fp,
                                               const DPart& cp, int tile, int gu, int gv,
                                               double* __restrict__ ccoef,
                                               float* __restrict__ ccoef32) {
  constexpr int dd = D < 0 ? 0 : D;
  constexpr int d1 = dd == 0 ? 1 : 0, d2 = dd == 2 ? 1 : 2;
  // the group's coarse entries (c = -1, 0, 1) and fine entries (o_d = -1, 0, 1)
  int ce[3], fe[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    int o[3];
    o[dd] = c - 1;
    o[d1] = gu;
    o[d2] = gv;
    const int code = (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1);
    ce[c] = cp.slot[code];
    fe[c] = fp.slot[code];
  }
  if (ce[0] < 0 && ce[1] < 0 && ce[2] < 0) return;
  const int fstr[3] = {1, fp.n[0], fp.n[0] * fp.n[1]};
#pragma unroll 1
  for (int m = 0, cc = (tile - cp.blk0) * cp.cpt * SSAMG_BLOCK + (int)threadIdx.x;
       m < cp.cpt && cc < cp.ncell; ++m, cc += SSAMG_BLOCK) {
    int I[3];
    cell_coords(cp, cc, I[0], I[1], I[2]);
    double acc[3] = {0.0, 0.0, 0.0};
    // offsets off d* are fixed within the group
    const bool off_in = (unsigned)(I[d1] + gu) < (unsigned)fp.n[d1] &&
                        (unsigned)(I[d2] + gv) < (unsigned)fp.n[d2];
    if (D < 0) {
      const int fcell = (I[2] * fp.n[1] + I[1]) * fp.n[0] + I[0];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        if (fe[c] >= 0 && off_in && (unsigned)(I[dd] + c - 1) < (unsigned)fp.n[dd])
          acc[c] = coef_at(fp, F.coef, fe[c], fcell);
    } else if (off_in) {
      const int anchor = 2 * I[dd] + fp.par;
      const int cell0 = (I[2] * fp.n[1] + I[1]) * fp.n[0] + I[0] + (anchor - I[dd]) * fstr[dd];
      // fine-point index of (f with coordinate x along d*, g off d*): the
      // fine-point grid halves d* only
      int q[3] = {I[0], I[1], I[2]};
      q[d1] += gu;
      q[d2] += gv;
      const int nfs[3] = {1, fp.nf[0], fp.nf[0] * fp.nf[1]};
      const int fp_off = fp.poff + q[d1] * nfs[d1] + q[d2] * nfs[d2];
      const int fpi0 = fp.poff + I[d1] * nfs[d1] + I[d2] * nfs[d2];
#pragma unroll
      for (int a = -1; a <= 1; ++a) {
        const int fd = anchor + a;
        if ((unsigned)fd >= (unsigned)fp.n[dd]) continue;
        const int fcell = cell0 + a * fstr[dd];
        double w1 = 1.0;
        if (a != 0) {
          const int Fi = fpi0 + ((fd + fp.par) >> 1) * nfs[dd];
          w1 = (a < 0) ? F.Pe[Fi] : F.Pw[Fi];
        }
        if (w1 == 0.0) continue;
#pragma unroll
        for (int od = -1; od <= 1; ++od) {
          const int e = fe[od + 1];
          const int gd = fd + od;
          if (e < 0 || (unsigned)gd >= (unsigned)fp.n[dd]) continue;
          const double v = w1 * coef_at(fp, F.coef, e, fcell);
          const int t = a + od;
          if ((t & 1) == 0) {
            acc[t / 2 + 1] += v;
          } else {
            const int Gi = fp_off + ((gd + fp.par) >> 1) * nfs[dd];
            acc[(t - 1) / 2 + 1] += v * F.Pw[Gi];
            acc[(t + 1) / 2 + 1] += v * F.Pe[Gi];
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (ce[c] < 0) continue;
      int O[3];
      O[dd] = c - 1;
      O[d1] = gu;
      O[d2] = gv;
      const double v = inside(cp, I[0] + O[0], I[1] + O[1], I[2] + O[2]) ? acc[c] : 0.0;
      ccoef[cp.coef[ce[c]] + cc] = v;
      if (ccoef32) ccoef32[cp.coef[ce[c]] + cc] = (float)v;
    }
  }
}

__global__ void __launch_bounds__(NT) k_rap_group(LevelView<double> F, LevelView<double> C,
                                                  double* __restrict__ ccoef,
                                                  float* __restrict__ ccoef32) {
  __shared__ DPart fp;
  __shared__ DPart cp;
  const int tile = (int)blockIdx.x / 9;
  const int grp = (int)blockIdx.x - 9 * tile;
  int p = block_part(C.blk, C.parts, C.np, cp, tile);
  part_of(F.parts, p, fp);
  __syncthreads();
  const int gu = grp % 3 - 1, gv = grp / 3 - 1;
  switch (fp.dstar) {
    case 0: rap_group_tile<0>(F, fp, cp, tile, gu, gv, ccoef, ccoef32); break;
    case 1: rap_group_tile<1>(F, fp, cp, tile, gu, gv, ccoef, ccoef32); break;
    case 2: rap_group_tile<2>(F, fp, cp, tile, gu, gv, ccoef, ccoef32); break;
    default: rap_group_tile<-1>(F, fp, cp, tile, gu, gv, ccoef, ccoef32); break;
  }
}

// ---------------------------------------------------------------------------
// K4: unstructured Galerkin product P^T U P (Eq. galerkin, second term).
// Rows of U_c are the coarse cells in the P-support of fine U rows (marker +
// scan); each coarse row gathers the U rows of its <= 3 fine points, spreads
// every entry over the column's P row, sorts by column and sums duplicates.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void locate(const LevelView<double>& L, const DPart* parts, int g,
                                       int& p, int& i, int& j, int& k) {
  p = find_part_cell(L.cellstart, L.np, g);
  const DPart& dp = parts[p];
  int c = g - dp.off;
  unsigned q = fdiv((unsigned)c, dp.dx);
  i = c - (int)q * dp.n[0];
  k = (int)fdiv((unsigned)c, dp.dxy);
  j = (int)q - k * dp.n[1];
}

// P's row at the cell of every fine coupling row r (Section 3.2): up to two
// coarse columns I with weights P(f, I) and the position a of f relative to
// I's anchor along d* (a = 0: f is I's coarse point or its part is not
// coarsened; +1: I is f's west neighbour; -1: its east neighbour), and the
// marker of the coarse rows of U_c.  Either output may be null: the marker
// alone needs no weights (it is taken before the level's interpolation).
__global__ void k_uprow(LevelView<double> F, int nr, const int* __restrict__ rows,
                        int* __restrict__ prI, double* __restrict__ prW,
                        signed char* __restrict__ prA, int* __restrict__ marker) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nr) return;
  int p, i, j, k;
  locate(F, F.parts, rows[r], p, i, j, k);
  const DPart& fp = F.parts[p];
  int I[2] = {-1, -1};
  double w[2] = {0.0, 0.0};
  signed char a[2] = {0, 0};
  const int d = fp.dstar;
  if (d < 0) {
    I[0] = coarse_index(fp, i, j, k);
    w[0] = 1.0;
  } else {
    const int cd = d == 0 ? i : (d == 1 ? j : k);
    auto at = [&](int v) {
      return coarse_index(fp, d == 0 ? v : i, d == 1 ? v : j, d == 2 ? v : k);
    };
    if (((cd + fp.par) & 1) == 0) {
      I[0] = at((cd - fp.par) >> 1);
      w[0] = 1.0;
    } else {
      const int Fi = fp.poff + fine_point_index(fp, i, j, k);
      if (cd - 1 >= 0) {
        I[0] = at((cd - 1 - fp.par) >> 1);
        if (prW) w[0] = F.Pw[Fi];
        a[0] = 1;
      }
      if (cd + 1 < fp.n[d]) {
        I[1] = at((cd + 1 - fp.par) >> 1);
        if (prW) w[1] = F.Pe[Fi];
        a[1] = -1;
      }
    }
  }
  for (int t = 0; t < 2; ++t) {
    if (prI) {
      prI[2 * r + t] = I[t];
      prW[2 * r + t] = w[t];
      prA[2 * r + t] = a[t];
    }
    if (marker && I[t] >= 0) marker[I[t]] = 1;
  }
}

// The (at most three) fine coupling rows of each coarse row of U_c, by their
// position a + 1 along d*, with their weights P(f, I).
__global__ void k_frows(int nr, const int* __restrict__ prI, const double* __restrict__ prW,
                        const signed char* __restrict__ prA, const int* __restrict__ cu_map,
                        int* __restrict__ fr, double* __restrict__ frw) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nr) return;
  for (int t = 0; t < 2; ++t) {
    const int I = prI[2 * r + t];
    if (I < 0) continue;
    const int R = cu_map[I];
    const int slot = 3 * R + prA[2 * r + t] + 1;
    fr[slot] = r;
    frw[slot] = prW[2 * r + t];
  }
}

__global__ void k_urows(int Nc, const int* __restrict__ scan, const int* __restrict__ marker_flag,
                        int* __restrict__ u_map, int* __restrict__ u_rows) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Nc) return;
  // marker_flag is the inclusive-minus-exclusive difference: scan[g+1] - scan[g]
  int s = scan[g];
  if (scan[g + 1] != s) {
    u_map[g] = s;
    u_rows[s] = g;
  } else {
    u_map[g] = -1;
  }
}

// Coarse row R of U_c = P^T U P, one warp per row.  The warp gathers the
// U rows of the coarse cell's fine points (at most 3 along d*, from the
// fine-row table fr, in the order a = -1, 0, +1), spreads every entry u_fg
// over P's row of g (at most 2 columns J, precomputed per coupling in pj, pw)
// into shared memory as candidates t = 0, 1, ... (generation order), sorts
// the keys (J, t) with a bitonic network, and merges equal columns: each run
// of equal J is one entry of the row, its slot the number of runs before it
// (columns ascending), its value the sum of the run's candidates in
// generation order (t ascending), so the result does not depend on the
// warp's schedule.  Instantiated with UW = 128 candidates per warp and 8
// warps per block for the rows whose candidate bound 2 sum_f len(f) is at
// most 128; longer rows go to the block form (k_urow_blk).
constexpr int UW_SMALL = 128, UWARPS_SMALL = 8;
constexpr int UW_LARGE = 1024;  // candidates of a row in the block form (k_urow_blk)

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int& total) {
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// Rows of at most UT candidates, one thread per row: the same candidates in
// the same generation order, sorted by (J, t) by insertion in the thread's
// own arrays, merged into runs of equal J summed in generation order, so the
// result is bitwise the warp form's.  Longer rows go to the warp forms: the
// thread lists them in midrows (midrows[0] = number).
//
// Every form sorts a row once: it reserves as many staging slots as the row
// has candidates (a bound on its entries; sum over rows <= 4 nnz of the fine
// level), writes the merged entries there (toff[R]: the first slot) and their
// number to counts[R]; k_ucopy moves them to the CSR arrays once the counts
// are scanned.  The staging order depends on the schedule, the result does not.
constexpr int UT = 16;
__global__ void __launch_bounds__(256) k_urow_t(LevelView<double> F, int nrc,
                                                int* __restrict__ midrows,
                                                const int* __restrict__ fr,
                                                const double* __restrict__ frw,
                                                const int* __restrict__ pj,
                                                const double* __restrict__ pw,
                                                int* __restrict__ counts, int* __restrict__ toff,
                                                int* __restrict__ cursor, int* __restrict__ tcol,
                                                double* __restrict__ tval,
                                                unsigned char* __restrict__ tbits) {
  const int R = blockIdx.x * blockDim.x + threadIdx.x;
  if (R >= nrc) return;
  int ur[3], q0[3], q1[3];
  double w1[3];
  int ub = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ur[a] = fr[3 * R + a];
    w1[a] = ur[a] >= 0 ? frw[3 * R + a] : 0.0;
    q0[a] = q1[a] = 0;
    if (ur[a] >= 0) {
      q0[a] = F.u_ptr[ur[a]];
      q1[a] = F.u_ptr[ur[a] + 1];
      ub += 2 * (q1[a] - q0[a]);
    }
  }
  if (ub > UT) {
    midrows[1 + atomicAdd(midrows, 1)] = R;
    return;
  }
  unsigned long long K[UT];
  double V[UT];
  unsigned char B[UT];
  int n = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    for (int q = q0[a]; q < q1[a]; ++q) {
      const double v = w1[a] * F.u_val[q];
      const unsigned char b = F.u_bits[q];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int J = pj[2 * q + t];
        if (J >= 0) {
          K[n] = ((unsigned long long)(unsigned)J << 10) | (unsigned)n;
          V[n] = v * pw[2 * q + t];
          B[n] = b;
          ++n;
        }
      }
    }
  for (int i = 1; i < n; ++i) {
    const unsigned long long key = K[i];
    int j = i - 1;
    while (j >= 0 && K[j] > key) {
      K[j + 1] = K[j];
      --j;
    }
    K[j + 1] = key;
  }
  const int o0 = n ? atomicAdd(cursor, n) : 0;
  int run = 0;
  for (int i = 0; i < n;) {
    const unsigned long long J = K[i] >> 10;
    double v = 0.0;
    unsigned char b = 0;
    int u = i;
    for (; u < n && (K[u] >> 10) == J; ++u) {
      const int t = (int)(K[u] & 1023ull);
      v += V[t];
      b |= B[t];
    }
    tcol[o0 + run] = (int)J;
    tval[o0 + run] = v;
    tbits[o0 + run] = b;
    ++run;
    i = u;
  }
  toff[R] = o0;
  counts[R] = run;
}

template <int UW, int WPB>
__global__ void __launch_bounds__(32 * WPB) k_urow(LevelView<double> F, int nrc,
                                                   const int* __restrict__ midrows,
                                                   int* __restrict__ longrows,
                                                   const int* __restrict__ fr,
                                                   const double* __restrict__ frw,
                                                   const int* __restrict__ pj,
                                                   const double* __restrict__ pw,
                                                   int* __restrict__ counts,
                                                   int* __restrict__ toff,
                                                   int* __restrict__ cursor,
                                                   int* __restrict__ tcol,
                                                   double* __restrict__ tval,
                                                   unsigned char* __restrict__ tbits,
                                                   int* __restrict__ err) {
  __shared__ unsigned long long sK[WPB][UW];
  __shared__ double sV[WPB][UW];
  __shared__ unsigned char sB[WPB][UW];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // both instances are fixed grids over a list of rows (list[0] = number,
  // then the rows): the small one over the rows the thread form left
  // (midrows), listing the rows it leaves to the large one (longrows); the
  // large one over longrows
  // (midrows null: the small one walks every row instead)
  constexpr bool small = UW == UW_SMALL;
  const int* list = small ? midrows : longrows;
  const int nlist = list ? *(volatile const int*)list : nrc;
  for (int it = blockIdx.x * WPB + w; it < nlist; it += gridDim.x * WPB) {
  const int R = list ? list[1 + it] : it;
  unsigned long long* K = sK[w];
  double* V = sV[w];
  unsigned char* B = sB[w];
  int ur[3], q0[3], q1[3];
  double w1[3];
  int ub = 0;
  for (int a = 0; a < 3; ++a) {
    ur[a] = fr[3 * R + a];
    w1[a] = ur[a] >= 0 ? frw[3 * R + a] : 0.0;
    q0[a] = q1[a] = 0;
    if (ur[a] >= 0) {
      q0[a] = F.u_ptr[ur[a]];
      q1[a] = F.u_ptr[ur[a] + 1];
      ub += 2 * (q1[a] - q0[a]);
    }
  }
  if (small && ub > UW_SMALL) {
    if (lane == 0) longrows[1 + atomicAdd(longrows, 1)] = R;
    continue;
  }
  int n = 0;
  for (int a = 0; a < 3; ++a) {
    if (ur[a] < 0) continue;
    for (int base = q0[a]; base < q1[a]; base += 32) {
      const int q = base + lane;
      int Jt[2] = {-1, -1};
      double w2[2] = {0.0, 0.0};
      double u = 0.0;
      unsigned char b = 0;
      if (q < q1[a]) {
        Jt[0] = pj[2 * q];
        Jt[1] = pj[2 * q + 1];
        w2[0] = pw[2 * q];
        w2[1] = pw[2 * q + 1];
        u = F.u_val[q];
        b = F.u_bits[q];
      }
      const int m = (Jt[0] >= 0) + (Jt[1] >= 0);
      int tot;
      int pos = n + warp_excl_scan(m, lane, tot);
      if (q < q1[a]) {
        const double v = w1[a] * u;
        for (int t = 0; t < 2; ++t)
          if (Jt[t] >= 0) {
            if (pos < UW) {
              K[pos] = ((unsigned long long)(unsigned)Jt[t] << 10) | (unsigned)pos;
              V[pos] = v * w2[t];
              B[pos] = b;
            }
            ++pos;
          }
      }
      n += tot;
    }
  }
  if (n > UW) {
    if (lane == 0) {
      atomicOr(err, 1);
      counts[R] = 0;
      toff[R] = 0;
    }
    continue;
  }
  // bitonic sort of the keys (padded to a power of two with the largest key)
  int m = 32;
  while (m < n) m <<= 1;
  for (int t = n + lane; t < m; t += 32) K[t] = ~0ull;
  __syncwarp();
  for (int k = 2; k <= m; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < m; i += 32) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long a = K[i], b = K[l];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            K[i] = b;
            K[l] = a;
          }
        }
      }
      __syncwarp();
    }
  // runs of equal columns: starts, their number and their staging slots
  int o0 = 0;
  if (lane == 0 && n) o0 = atomicAdd(cursor, n);
  o0 = __shfl_sync(0xffffffffu, o0, 0);
  int run = 0;
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    const bool start = i < n && (i == 0 || (K[i] >> 10) != (K[i - 1] >> 10));
    int tot;
    const int slot = run + warp_excl_scan(start ? 1 : 0, lane, tot);
    if (start) {
      const unsigned long long J = K[i] >> 10;
      double v = 0.0;
      unsigned char b = 0;
      for (int u = i; u < n && (K[u] >> 10) == J; ++u) {
        const int t = (int)(K[u] & 1023ull);
        v += V[t];
        b |= B[t];
      }
      tcol[o0 + slot] = (int)J;
      tval[o0 + slot] = v;
      tbits[o0 + slot] = b;
    }
    run += tot;
  }
  if (lane == 0) {
    counts[R] = run;
    toff[R] = o0;
  }
  __syncwarp();
  }
}

// Block-wide exclusive scan of one int per thread (NTB threads); total in
// `total`.  All threads must call.
template <int NTB>
__device__ __forceinline__ int block_excl_scan(int v, int* sh, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < NTB / 32 ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < NTB / 32) sh[lane] = t;  // inclusive warp-total prefix
  }
  __syncthreads();
  total = sh[NTB / 32 - 1];
  const int before = w > 0 ? sh[w - 1] : 0;
  __syncthreads();
  return before + x - v;
}

// Rows of more than UW_SMALL candidates (up to UW_LARGE), a block of NTB
// threads per row: the same candidates in the same generation order (the
// positions by a block scan over the entries' candidate counts), the same
// keys (J, t) sorted by a bitonic network over the whole block, the same
// runs summed in generation order by their first thread: bitwise the warp
// form's rows, with the sort's stages spread over NTB threads instead of 32.
constexpr int UBLK = 256;
__global__ void __launch_bounds__(UBLK) k_urow_blk(LevelView<double> F,
                                                   const int* __restrict__ longrows,
                                                   const int* __restrict__ fr,
                                                   const double* __restrict__ frw,
                                                   const int* __restrict__ pj,
                                                   const double* __restrict__ pw,
                                                   int* __restrict__ counts,
                                                   int* __restrict__ toff,
                                                   int* __restrict__ cursor,
                                                   int* __restrict__ tcol,
                                                   double* __restrict__ tval,
                                                   unsigned char* __restrict__ tbits,
                                                   int* __restrict__ err) {
  __shared__ unsigned long long K[UW_LARGE];
  __shared__ double V[UW_LARGE];
  __shared__ unsigned char B[UW_LARGE];
  __shared__ int sh[UBLK / 32];
  __shared__ int s_o0;
  const int tid = threadIdx.x;
  const int nlist = *(volatile const int*)longrows;
  for (int it = blockIdx.x; it < nlist; it += gridDim.x) {
    const int R = longrows[1 + it];
    int ur[3], q0[3], q1[3];
    double w1[3];
    for (int a = 0; a < 3; ++a) {
      ur[a] = fr[3 * R + a];
      w1[a] = ur[a] >= 0 ? frw[3 * R + a] : 0.0;
      q0[a] = q1[a] = 0;
      if (ur[a] >= 0) {
        q0[a] = F.u_ptr[ur[a]];
        q1[a] = F.u_ptr[ur[a] + 1];
      }
    }
    int n = 0;
    for (int a = 0; a < 3; ++a) {
      if (ur[a] < 0) continue;
      for (int base = q0[a]; base < q1[a]; base += UBLK) {
        const int q = base + tid;
        int Jt[2] = {-1, -1};
        double w2[2] = {0.0, 0.0};
        double u = 0.0;
        unsigned char b = 0;
        if (q < q1[a]) {
          Jt[0] = pj[2 * q];
          Jt[1] = pj[2 * q + 1];
          w2[0] = pw[2 * q];
          w2[1] = pw[2 * q + 1];
          u = F.u_val[q];
          b = F.u_bits[q];
        }
        const int m = (Jt[0] >= 0) + (Jt[1] >= 0);
        int tot;
        int pos = n + block_excl_scan<UBLK>(m, sh, tot);
        if (q < q1[a]) {
          const double v = w1[a] * u;
          for (int t = 0; t < 2; ++t)
            if (Jt[t] >= 0) {
              if (pos < UW_LARGE) {
                K[pos] = ((unsigned long long)(unsigned)Jt[t] << 10) | (unsigned)pos;
                V[pos] = v * w2[t];
                B[pos] = b;
              }
              ++pos;
            }
        }
        n += tot;
      }
    }
    if (n > UW_LARGE) {
      if (tid == 0) {
        atomicOr(err, 1);
        counts[R] = 0;
        toff[R] = 0;
      }
      __syncthreads();
      continue;
    }
    int m = 32;
    while (m < n) m <<= 1;
    for (int t = n + tid; t < m; t += UBLK) K[t] = ~0ull;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < m; i += UBLK) {
          const int l = i ^ j;
          if (l > i) {
            const unsigned long long x = K[i], y = K[l];
            if ((x > y) == ((i & k) == 0)) {
              K[i] = y;
              K[l] = x;
            }
          }
        }
        __syncthreads();
      }
    if (tid == 0) s_o0 = n ? atomicAdd(cursor, n) : 0;
    __syncthreads();
    const int o0 = s_o0;
    int run = 0;
    for (int base = 0; base < n; base += UBLK) {
      const int i = base + tid;
      const bool start = i < n && (i == 0 || (K[i] >> 10) != (K[i - 1] >> 10));
      int tot;
      const int slot = run + block_excl_scan<UBLK>(start ? 1 : 0, sh, tot);
      if (start) {
        const unsigned long long J = K[i] >> 10;
        double v = 0.0;
        unsigned char b = 0;
        for (int u = i; u < n && (K[u] >> 10) == J; ++u) {
          const int t = (int)(K[u] & 1023ull);
          v += V[t];
          b |= B[t];
        }
        tcol[o0 + slot] = (int)J;
        tval[o0 + slot] = v;
        tbits[o0 + slot] = b;
      }
      run += tot;
    }
    if (tid == 0) {
      counts[R] = run;
      toff[R] = o0;
    }
    __syncthreads();
  }
}

// For every coupling q of level l: the coarse columns and weights of P's row
// of its column cell (used by the prolongation's row jobs).
__device__ __forceinline__ void upcol(const LevelView<double>& F, long long q,
                                      int* __restrict__ pj, double* __restrict__ pw,
                                      float* __restrict__ pw32) {
  int gq, gi, gj, gk;
  locate(F, F.parts, F.u_col[q], gq, gi, gj, gk);
  int J[2] = {-1, -1};
  double w[2] = {0.0, 0.0};
  p_row_arrays(F.parts[gq], F.Pw, F.Pe, gi, gj, gk, J, w);
  for (int t = 0; t < 2; ++t) {
    pj[2 * q + t] = J[t];
    pw[2 * q + t] = w[t];
    if (pw32) pw32[2 * q + t] = (float)w[t];
  }
}

// Restriction row of each coupling's column cell on a coarse level: the
// fine cells (centre, -d*, +d* neighbours; -1 absent) and the side weights
// (PE of the -d* fine point, PW of the +d*), as the restriction applies them.
__device__ __forceinline__ void urcol_at(const LevelView<double>& F, const LevelView<double>& C,
                                         int col, long long q, int* __restrict__ rj,
                                         double* __restrict__ rw, float* __restrict__ rw32) {
  int p, I[3];
  locate(C, C.parts, col, p, I[0], I[1], I[2]);
  const DPart& fp = F.parts[p];
  const int d = fp.dstar;
  int j0, j1 = -1, j2 = -1;
  double w1 = 0.0, w2 = 0.0;
  if (d < 0) {
    j0 = fp.off + (I[2] * fp.n[1] + I[1]) * fp.n[0] + I[0];
  } else {
    int f[3] = {I[0], I[1], I[2]};
    const int anchor = 2 * I[d] + fp.par;
    f[d] = anchor;
    const int sd = (d == 0) ? 1 : (d == 1 ? fp.n[0] : fp.n[0] * fp.n[1]);
    j0 = fp.off + (f[2] * fp.n[1] + f[1]) * fp.n[0] + f[0];
    if (anchor - 1 >= 0) {
      f[d] = anchor - 1;
      j1 = j0 - sd;
      w1 = F.Pe[fp.poff + fine_point_index(fp, f[0], f[1], f[2])];
    }
    if (anchor + 1 < fp.n[d]) {
      f[d] = anchor + 1;
      j2 = j0 + sd;
      w2 = F.Pw[fp.poff + fine_point_index(fp, f[0], f[1], f[2])];
    }
  }
  rj[3 * q] = j0;
  rj[3 * q + 1] = j1;
  rj[3 * q + 2] = j2;
  rw[2 * q] = w1;
  rw[2 * q + 1] = w2;
  if (rw32) {
    rw32[2 * q] = (float)w1;
    rw32[2 * q + 1] = (float)w2;
  }
}

__device__ __forceinline__ void urcol(const LevelView<double>& F, const LevelView<double>& C,
                                      long long q, int* __restrict__ rj, double* __restrict__ rw,
                                      float* __restrict__ rw32) {
  urcol_at(F, C, C.u_col[q], q, rj, rw, rw32);
}

// Setup data of a level's row jobs, per coupling: P's row of its column cell
// (with pj: the prolongation's U x) and its restriction row from the level
// above (with rj: the pre-relaxation fused into the restriction onto it).
__global__ void k_ucols(LevelView<double> Fp, LevelView<double> L, long long nnz,
                        int* __restrict__ pj, double* __restrict__ pw, float* __restrict__ pw32,
                        int* __restrict__ rj, double* __restrict__ rw, float* __restrict__ rw32) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nnz) return;
  if (pj) upcol(L, q, pj, pw, pw32);
  if (rj) urcol(Fp, L, q, rj, rw, rw32);
}

// ---------------------------------------------------------------------------
// K5: diagonal of omega M^-1 (Section 3.4).
// ---------------------------------------------------------------------------
// Every level's smoother diagonal in one launch: block b works on the level
// whose block range holds it (the levels' tile grids one after another).
struct DinvLevel {
  const DPart* parts;
  const int* blk;
  const double* coef;
  const int* u_map;
  const int* u_ptr;
  const double* u_val;
  double* dinv;
  float* dinv32;
  int np;
  int b0;  // first block of the level in the launch
};
struct DinvArgs {
  int nl;
  int relax;
  double factor;
  DinvLevel lv[SSAMG_DINV_LEVELS];
};

__global__ void __launch_bounds__(NT) k_dinv(const __grid_constant__ DinvArgs A) {
  __shared__ DPart sp;
  int l = 0;
  while (l + 1 < A.nl && (int)blockIdx.x >= A.lv[l + 1].b0) ++l;
  const DinvLevel& L = A.lv[l];
  const int tile = (int)blockIdx.x - L.b0;
  block_part(L.blk, L.parts, L.np, sp, tile);
  __syncthreads();
#pragma unroll 1
  for (int m = 0, c = (tile - sp.blk0) * sp.cpt * SSAMG_BLOCK + (int)threadIdx.x;
       m < sp.cpt && c < sp.ncell; ++m, c += SSAMG_BLOCK) {
    int i, j, k;
    cell_coords(sp, c, i, j, k);
    double v;
    if (A.relax == 0) {
      double diag = 0.0;
      for (int e = 0; e < sp.nent; ++e)
        if (sp.o[e][0] == 0 && sp.o[e][1] == 0 && sp.o[e][2] == 0) diag += coef_at(sp, L.coef, e, c);
      double w = A.factor > 0.0 ? A.factor : sp.omega;
      v = w / diag;
    } else {
      double s = 0.0;
      for (int e = 0; e < sp.nent; ++e)
        if (inside(sp, i + sp.o[e][0], j + sp.o[e][1], k + sp.o[e][2]))
          s += fabs(coef_at(sp, L.coef, e, c));
      if (sp.has_u) {
        int r = L.u_map[sp.off + c];
        if (r >= 0)
          for (int q = L.u_ptr[r]; q < L.u_ptr[r + 1]; ++q) s += fabs(L.u_val[q]);
      }
      double w = A.factor > 0.0 ? A.factor : 1.5;
      v = w / s;
    }
    if (sp.skip) v = 0.0;  // relaxation turned off: omega M^-1 = 0
    L.dinv[sp.off + c] = v;
    if (L.dinv32) L.dinv32[sp.off + c] = (float)v;
  }
}

__global__ void k_mask_outside(double* __restrict__ v, int nx, int ny, int nz, int ox, int oy,
                               int oz) {
  long long n = (long long)nx * ny * nz;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    if ((unsigned)(i + ox) >= (unsigned)nx || (unsigned)(j + oy) >= (unsigned)ny ||
        (unsigned)(k + oz) >= (unsigned)nz)
      v[c] = 0.0;
  }
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, long long n) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; t < n; t += (long long)gridDim.x * blockDim.x) out[t] = (float)in[t];
}

// ---------------------------------------------------------------------------
// Coarsest level: dense assembly and Cholesky (FP64).
// ---------------------------------------------------------------------------
__global__ void k_coarse_assemble(LevelView<double> L, double* __restrict__ A) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.N) return;
  int p = find_part_cell(L.cellstart, L.np, g);
  const DPart& dp = L.parts[p];
  int c = g - dp.off;
  int i, j, k;
  {
    unsigned q = fdiv((unsigned)c, dp.dx);
    i = c - (int)q * dp.n[0];
    k = (int)fdiv((unsigned)c, dp.dxy);
    j = (int)q - k * dp.n[1];
  }
  double* row = A + (long long)g * L.N;
  for (int t = 0; t < L.N; ++t) row[t] = 0.0;
  for (int e = 0; e < dp.nent; ++e) {
    if (!inside(dp, i + dp.o[e][0], j + dp.o[e][1], k + dp.o[e][2])) continue;
    row[g + dp.disp[e]] += coef_at(dp, L.coef, e, c);
  }
  if (dp.has_u) {
    int r = L.u_map[g];
    if (r >= 0)
      for (int q = L.u_ptr[r]; q < L.u_ptr[r + 1]; ++q) row[L.u_col[q]] += L.u_val[q];
  }
}

// Left-looking Cholesky A = L L^T in place (lower triangle), one block.
// status: 0 ok, 1 not positive definite.
__global__ void __launch_bounds__(NT) k_cholesky(int n, double* __restrict__ A, int* status) {
  __shared__ double sh[NT];
  __shared__ double piv;
  for (int jj = 0; jj < n; ++jj) {
    double* rj = A + (long long)jj * n;
    double s = 0.0;
    for (int k = threadIdx.x; k < jj; k += NT) s += rj[k] * rj[k];
    double tot = block_sum<NT>(s, sh);
    if (threadIdx.x == 0) {
      double dd = rj[jj] - tot;
      if (!(dd > 0.0)) {
        *status = 1;
        dd = 1.0;
      }
      piv = sqrt(dd);
      rj[jj] = piv;
    }
    __syncthreads();
    for (int i = jj + 1 + threadIdx.x; i < n; i += NT) {
      double* ri = A + (long long)i * n;
      double t = ri[jj];
      for (int k = 0; k < jj; ++k) t -= ri[k] * rj[k];
      ri[jj] = t / piv;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Exclusive scan of ints (three passes; data[n] receives the total).
// ---------------------------------------------------------------------------
constexpr int SCAN_ITEMS = 1024;

__global__ void __launch_bounds__(NT) k_scan_reduce(const int* __restrict__ in, long long n,
                                                    int* __restrict__ sums) {
  __shared__ int sh[NT];
  long long base = (long long)blockIdx.x * SCAN_ITEMS;
  int s = 0;
  for (int t = threadIdx.x; t < SCAN_ITEMS; t += NT)
    if (base + t < n) s += in[base + t];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(1024) k_scan_sums(int* __restrict__ sums, int nb) {
  // single block: exclusive scan of nb block sums, sums[nb] = total
  __shared__ int sh[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    int t = base + threadIdx.x;
    int v = t < nb ? sums[t] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int u = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += u;
      __syncthreads();
    }
    if (t < nb) sums[t] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

// Block b scans items [b SCAN_ITEMS, (b+1) SCAN_ITEMS) in parallel (four
// consecutive items per thread, shuffle scan of the thread sums, then the
// warp sums) and adds the block's offset sums[b] (0 without sums: the
// single-block case).  The last block writes the total to data[n].
__global__ void __launch_bounds__(NT) k_scan_apply(int* __restrict__ data, long long n,
                                                   const int* __restrict__ sums, int nb) {
  static_assert(SCAN_ITEMS == 4 * NT, "four items per thread");
  __shared__ int sh[SCAN_ITEMS];
  __shared__ int wsum[NT / 32];
  const long long base = (long long)blockIdx.x * SCAN_ITEMS;
  for (int t = threadIdx.x; t < SCAN_ITEMS; t += NT) sh[t] = base + t < n ? data[base + t] : 0;
  __syncthreads();
  const int t4 = 4 * (int)threadIdx.x;
  const int a0 = sh[t4], a1 = sh[t4 + 1], a2 = sh[t4 + 2], a3 = sh[t4 + 3];
  const int own = a0 + a1 + a2 + a3;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = own;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int v = lane < NT / 32 ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane < NT / 32) wsum[lane] = v;  // inclusive warp totals
  }
  __syncthreads();
  const int off0 = sums ? sums[blockIdx.x] : 0;
  const int e = off0 + x - own + (w > 0 ? wsum[w - 1] : 0);
  sh[t4] = e;
  sh[t4 + 1] = e + a0;
  sh[t4 + 2] = e + a0 + a1;
  sh[t4 + 3] = e + a0 + a1 + a2;
  __syncthreads();
  for (int t = threadIdx.x; t < SCAN_ITEMS; t += NT)
    if (base + t < n) data[base + t] = sh[t];
  if (blockIdx.x == nb - 1 && threadIdx.x == 0)
    data[n] = sums ? sums[nb] : wsum[NT / 32 - 1];
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// The staged rows of U_c into its CSR arrays (ptr: the scanned counts), a
// warp per row, and with every entry its restriction row from the level
// above (the row jobs' data for the pre-relaxation fused into the
// restriction, as k_ucols makes it).
__global__ void __launch_bounds__(256) k_ucopy(LevelView<double> F, LevelView<double> C, int nr,
                                               const int* __restrict__ ptr,
                                               const int* __restrict__ toff,
                                               const int* __restrict__ tcol,
                                               const double* __restrict__ tval,
                                               const unsigned char* __restrict__ tbits,
                                               int* __restrict__ col, double* __restrict__ val,
                                               float* __restrict__ val32,
                                               unsigned char* __restrict__ bits,
                                               int* __restrict__ rj, double* __restrict__ rw,
                                               float* __restrict__ rw32) {
  const int R = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (R >= nr) return;
  const int o = ptr[R], n = ptr[R + 1] - o, t = toff[R];
  for (int i = lane; i < n; i += 32) {
    const double v = tval[t + i];
    const int J = tcol[t + i];
    col[o + i] = J;
    val[o + i] = v;
    if (val32) val32[o + i] = (float)v;
    bits[o + i] = tbits[t + i];
    if (rj) urcol_at(F, C, J, o + i, rj, rw, rw32);
  }
}

// ---------------------------------------------------------------------------
// Level-0 coupling rows from the user's m (row, col, value, bits) tuples: a
// counting sort by row, then per row the entries ordered by (column, input
// position), equal columns summed in input order with their direction bits
// OR'ed; rows ascending, columns ascending within a row.
// ---------------------------------------------------------------------------
__global__ void k_ua_count(long long m, const int* __restrict__ row, int* __restrict__ cnt) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) atomicAdd(cnt + row[t], 1);
}

__global__ void k_ua_scatter(long long m, const int* __restrict__ row,
                             const int* __restrict__ start, int* __restrict__ fill,
                             int* __restrict__ perm) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const int r = row[t];
  perm[start[r] + atomicAdd(fill + r, 1)] = (int)t;
}

__global__ void k_ua_rows(int N, const int* __restrict__ start, int* __restrict__ perm,
                          const int* __restrict__ col, int* __restrict__ uniq,
                          int* __restrict__ flag) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  const int s0 = start[g], n = start[g + 1] - s0;
  if (n == 0) {
    uniq[g] = 0;
    flag[g] = 0;
    return;
  }
  int* pr = perm + s0;
  // insertion sort by (column, input position): rows hold a few entries
  for (int i = 1; i < n; ++i) {
    const int t = pr[i], ct = col[t];
    int j = i - 1;
    while (j >= 0 && (col[pr[j]] > ct || (col[pr[j]] == ct && pr[j] > t))) {
      pr[j + 1] = pr[j];
      --j;
    }
    pr[j + 1] = t;
  }
  int u = 1;
  for (int i = 1; i < n; ++i) u += col[pr[i]] != col[pr[i - 1]];
  uniq[g] = u;
  flag[g] = 1;
}

__global__ void k_ua_fill(int N, const int* __restrict__ start, const int* __restrict__ perm,
                          const int* __restrict__ col, const double* __restrict__ val,
                          const unsigned char* __restrict__ bits, const int* __restrict__ uoff,
                          const int* __restrict__ roff, int* __restrict__ u_rows,
                          int* __restrict__ u_ptr, int* __restrict__ u_col,
                          double* __restrict__ u_val, unsigned char* __restrict__ u_bits,
                          int* __restrict__ u_map) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g == 0) u_ptr[roff[N]] = uoff[N];
  if (g >= N) return;
  const int r = roff[g];
  if (roff[g + 1] == r) {
    u_map[g] = -1;
    return;
  }
  u_map[g] = r;
  u_rows[r] = g;
  int q = uoff[g];
  u_ptr[r] = q;
  const int s0 = start[g], s1 = start[g + 1];
  for (int i = s0; i < s1;) {
    const int c = col[perm[i]];
    double v = 0.0;
    unsigned char b = 0;
    for (; i < s1 && col[perm[i]] == c; ++i) {
      v += val[perm[i]];
      b |= bits[perm[i]];
    }
    u_col[q] = c;
    u_val[q] = v;
    u_bits[q] = b;
    ++q;
  }
}

__device__ __forceinline__ bool in_boxes(const PartBoxes& pb, int i, int j, int k) {
  for (int b = 0; b < pb.n; ++b)
    if (i >= pb.b[b][0] && i <= pb.b[b][3] && j >= pb.b[b][1] && j <= pb.b[b][4] &&
        k >= pb.b[b][2] && k <= pb.b[b][5])
      return true;
  return false;
}

__global__ void k_mask_part(double* __restrict__ v, int nx, int ny, int nz, int ox, int oy, int oz,
                            const __grid_constant__ PartBoxes pb) {
  const long long n = (long long)nx * ny * nz;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % nx), j = (int)((c / nx) % ny), k = (int)(c / ((long long)nx * ny));
    const bool act = in_boxes(pb, i, j, k);
    if (ox == 0 && oy == 0 && oz == 0) {
      if (!act) v[c] = 1.0;
    } else if (!act || !in_boxes(pb, i + ox, j + oy, k + oz)) {
      v[c] = 0.0;
    }
  }
}


}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Block partials of the allocation-free coupling sums: one triple per block
// of a level launch, every slot written before it is read.
static __device__ __align__(256) double g_wsum_scratch[3 * SSAMG_NOALLOC_MAX_BLOCKS];

double* wsum_static_scratch() {
  void* p = nullptr;
  SSAMG_CUDA(cudaGetSymbolAddress(&p, g_wsum_scratch));
  return static_cast<double*>(p);
}

void launch_wsum(const Level& L, double* partial, double* c_out, cudaStream_t st) {
  k_wsum<<<L.nblk, NT, 0, st>>>(L.view<double>(), partial);
  SSAMG_LAUNCH_CHECK();
  k_wfinal<<<L.np, NT, 0, st>>>(L.d_blk, partial, c_out);
  SSAMG_LAUNCH_CHECK();
}

void launch_interp(const Level& F, bool fp32, cudaStream_t st) {
  if (F.nfblk == 0) return;
  k_interp<<<F.nfblk, NT, 0, st>>>(F.view<double>(), F.Pw, F.Pe, fp32 ? F.Pw32 : nullptr,
                                   fp32 ? F.Pe32 : nullptr);
  SSAMG_LAUNCH_CHECK();
}

void launch_rap_struct(const Level& F, const Level& Cl, bool fp32, cudaStream_t st) {
  k_rap_group<<<Cl.nblk * 9, NT, 0, st>>>(F.view<double>(), Cl.view<double>(), Cl.coef,
                                          fp32 ? Cl.coef32 : nullptr);
  SSAMG_LAUNCH_CHECK();
}

void launch_uprow(const Level& F, const Level& Cl, int* prI, double* prW, signed char* prA,
                  int* marker, cudaStream_t st) {
  if (marker) SSAMG_CUDA(cudaMemsetAsync(marker, 0, sizeof(int) * (Cl.N + 1), st));
  if (F.nr > 0) {
    k_uprow<<<cdiv(F.nr, NT), NT, 0, st>>>(F.view<double>(), F.nr, F.u_rows, prI, prW, prA,
                                          marker);
    SSAMG_LAUNCH_CHECK();
  }
}

void launch_frows(const Level& F, const Level& Cl, const int* prI, const double* prW,
                  const signed char* prA, int* fr, double* frw, cudaStream_t st) {
  SSAMG_CUDA(cudaMemsetAsync(fr, 0xff, sizeof(int) * 3 * (size_t)std::max(Cl.nr, 1), st));
  if (F.nr > 0 && Cl.nr > 0) {
    k_frows<<<cdiv(F.nr, NT), NT, 0, st>>>(F.nr, prI, prW, prA, Cl.u_map, fr, frw);
    SSAMG_LAUNCH_CHECK();
  }
}

void launch_urows(const Level& Cl, const int* scan, const int* marker, cudaStream_t st) {
  k_urows<<<cdiv(Cl.N, NT), NT, 0, st>>>((int)Cl.N, scan, marker, Cl.u_map, Cl.u_rows);
  SSAMG_LAUNCH_CHECK();
}

// The three forms of the coupling-row merge: a thread per row of at most UT
// candidates over every row, then the warp forms (fixed grids of a few blocks
// per SM) over the rows the form before listed: midrows (more than UT
// candidates, up to UW_SMALL) and longrows (more than UW_SMALL).  lists:
// 2 (nr + 1) ints, midrows then longrows.
// The thread form runs first only where the fine level's coupling rows are
// short (mean length <= 8/3: three fine rows spread over two columns each
// then give at most 16 candidates on average); elsewhere the small warp form
// walks every row.
bool urow_thread_form(const Level& F) { return 3ll * F.nnz <= 8ll * F.nr; }

void launch_usort(const Level& F, const Level& Cl, int* lists, const int* fr,
                  const double* frw, int* counts, const UStage& t, int* err, cudaStream_t st) {
  if (Cl.nr == 0) return;
  const bool thr = urow_thread_form(F);
  int* midrows = thr ? lists : nullptr;
  int* longrows = lists + Cl.nr + 1;
  SSAMG_CUDA(cudaMemsetAsync(lists, 0, sizeof(int), st));
  SSAMG_CUDA(cudaMemsetAsync(longrows, 0, sizeof(int), st));
  SSAMG_CUDA(cudaMemsetAsync(t.cursor, 0, sizeof(int), st));
  int dev = 0, sms = 0;
  SSAMG_CUDA(cudaGetDevice(&dev));
  SSAMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (thr) {
    k_urow_t<<<cdiv(Cl.nr, 256), 256, 0, st>>>(F.view<double>(), Cl.nr, midrows, fr, frw,
                                                F.u_pj, F.u_pw, counts, t.toff, t.cursor,
                                                t.col, t.val, t.bits);
    SSAMG_LAUNCH_CHECK();
  }
  const int nbs = thr ? std::min(cdiv(Cl.nr, UWARPS_SMALL), 4 * sms) : cdiv(Cl.nr, UWARPS_SMALL);
  k_urow<UW_SMALL, UWARPS_SMALL><<<nbs, 32 * UWARPS_SMALL, 0, st>>>(
      F.view<double>(), Cl.nr, midrows, longrows, fr, frw, F.u_pj, F.u_pw, counts, t.toff,
      t.cursor, t.col, t.val, t.bits, err);
  SSAMG_LAUNCH_CHECK();
k_urow_blk<<<std::min(Cl.nr, 2 * sms), UBLK, 0, st>>>(F.view<double>(), longrows, fr, frw,
                                                        F.u_pj, F.u_pw, counts, t.toff, t.cursor,
                                                        t.col, t.val, t.bits, err);
  SSAMG_LAUNCH_CHECK();
}

void launch_ucopy(const Level& F, const Level& Cl, const UStage& t, bool fp32, cudaStream_t st) {
  if (Cl.nr == 0 || Cl.nnz == 0) return;
  k_ucopy<<<cdiv(Cl.nr, 8), 256, 0, st>>>(F.view<double>(), Cl.view<double>(), Cl.nr, Cl.u_ptr,
                                          t.toff, t.col, t.val, t.bits, Cl.u_col, Cl.u_val,
                                          fp32 ? Cl.u_val32 : nullptr, Cl.u_bits, Cl.u_rj,
                                          Cl.u_rw, fp32 ? Cl.u_rw32 : nullptr);
  SSAMG_LAUNCH_CHECK();
}

void launch_ucols(const Level* Fp, const Level& L, bool fp32, bool pj, bool rj, cudaStream_t st) {
  int* dpj = pj ? L.u_pj : nullptr;
  int* drj = rj ? L.u_rj : nullptr;
  if (L.nnz == 0 || (!dpj && !drj)) return;
  k_ucols<<<cdiv(L.nnz, NT), NT, 0, st>>>(Fp ? Fp->view<double>() : L.view<double>(),
                                         L.view<double>(), L.nnz, dpj, L.u_pw,
                                         fp32 ? L.u_pw32 : nullptr, drj, L.u_rw,
                                         fp32 ? L.u_rw32 : nullptr);
  SSAMG_LAUNCH_CHECK();
}


void launch_dinv(const std::vector<Level>& lev, int first, int last, int relax, double factor,
                 bool fp32, cudaStream_t st) {
  for (int l0 = first; l0 <= last; l0 += SSAMG_DINV_LEVELS) {
    DinvArgs a{};
    a.relax = relax;
    a.factor = factor;
    int nb = 0;
    for (int l = l0; l <= last && a.nl < SSAMG_DINV_LEVELS; ++l) {
      const Level& L = lev[l];
      a.lv[a.nl++] = DinvLevel{L.d_parts, L.d_blk, L.coef, L.u_map, L.u_ptr, L.u_val,
                               L.dinv, fp32 ? L.dinv32 : nullptr, L.np, nb};
      nb += L.nblk;
    }
    k_dinv<<<nb, NT, 0, st>>>(a);
    SSAMG_LAUNCH_CHECK();
  }
}

void launch_to_float(const double* in, float* out, long long n, cudaStream_t st) {
  if (n <= 0) return;
  int nb = (int)std::min<long long>(cdiv(n, NT), 152 * 16);
  k_to_float<<<nb, NT, 0, st>>>(in, out, n);
  SSAMG_LAUNCH_CHECK();
}

void launch_mask_outside(double* vals, const int n[3], const int o[3], cudaStream_t st) {
  long long cnt = (long long)n[0] * n[1] * n[2];
  int nb = (int)std::min<long long>(cdiv(cnt, NT), 152 * 8);
  k_mask_outside<<<nb, NT, 0, st>>>(vals, n[0], n[1], n[2], o[0], o[1], o[2]);
  SSAMG_LAUNCH_CHECK();
}

void launch_coarse_assemble(const Level& L, double* A, cudaStream_t st) {
  k_coarse_assemble<<<cdiv(L.N, 64), 64, 0, st>>>(L.view<double>(), A);
  SSAMG_LAUNCH_CHECK();
}

void launch_cholesky(int n, double* A, int* status, cudaStream_t st) {
  k_cholesky<<<1, NT, 0, st>>>(n, A, status);
  SSAMG_LAUNCH_CHECK();
}

size_t scan_tmp_ints(long long n) { return (size_t)cdiv(n, SCAN_ITEMS) + 1; }

void launch_scan(int* data, long long n, int* tmp, cudaStream_t st) {
  if (n <= 0) {
    SSAMG_CUDA(cudaMemsetAsync(data, 0, sizeof(int), st));
    return;
  }
  int nb = cdiv(n, SCAN_ITEMS);
  if (nb == 1) {  // one block scans it all
    k_scan_apply<<<1, NT, 0, st>>>(data, n, nullptr, 1);
    SSAMG_LAUNCH_CHECK();
    return;
  }
  k_scan_reduce<<<nb, NT, 0, st>>>(data, n, tmp);
  SSAMG_LAUNCH_CHECK();
  k_scan_sums<<<1, 1024, 0, st>>>(tmp, nb);
  SSAMG_LAUNCH_CHECK();
  k_scan_apply<<<nb, NT, 0, st>>>(data, n, tmp, nb);
  SSAMG_LAUNCH_CHECK();
}

void launch_uassemble(const UAssemble& a, int* nr, long long* nnz, cudaStream_t st) {
  const int N = a.N;
  int* cnt = (int*)pool_alloc(sizeof(int) * ((size_t)N + 1));
  int* fill = (int*)pool_alloc(sizeof(int) * (size_t)N);
  int* perm = (int*)pool_alloc(sizeof(int) * (size_t)a.m);
  int* uniq = (int*)pool_alloc(sizeof(int) * ((size_t)N + 1));
  int* flag = (int*)pool_alloc(sizeof(int) * ((size_t)N + 1));
  int* tmp = (int*)pool_alloc(sizeof(int) * (scan_tmp_ints((long long)N + 1) + 1));
  int* tot = (int*)pool_alloc(sizeof(int) * 2);
  if (!cnt || !fill || !perm || !uniq || !flag || !tmp || !tot) {
    pool_fence();
    for (void* q : {(void*)cnt, (void*)fill, (void*)perm, (void*)uniq, (void*)flag, (void*)tmp, (void*)tot})
      pool_free(q);
    throw SsamgError{SSAMG_ERR_OOM, "device allocation failed"};
  }
  SSAMG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)N + 1), st));
  SSAMG_CUDA(cudaMemsetAsync(fill, 0, sizeof(int) * (size_t)N, st));
  const int mb = cdiv(a.m, NT);
  k_ua_count<<<mb, NT, 0, st>>>(a.m, a.row, cnt);
  SSAMG_LAUNCH_CHECK();
  launch_scan(cnt, N, tmp, st);
  k_ua_scatter<<<mb, NT, 0, st>>>(a.m, a.row, cnt, fill, perm);
  SSAMG_LAUNCH_CHECK();
  k_ua_rows<<<cdiv(N, NT), NT, 0, st>>>(N, cnt, perm, a.col, uniq, flag);
  SSAMG_LAUNCH_CHECK();
  launch_scan(uniq, N, tmp, st);
  launch_scan(flag, N, tmp, st);
  k_ua_fill<<<cdiv(N, NT), NT, 0, st>>>(N, cnt, perm, a.col, a.val, a.bits, uniq, flag, a.u_rows,
                                        a.u_ptr, a.u_col, a.u_val, a.u_bits, a.u_map);
  SSAMG_LAUNCH_CHECK();
  SSAMG_CUDA(cudaMemcpyAsync(tot, flag + N, sizeof(int), cudaMemcpyDeviceToDevice, st));
  SSAMG_CUDA(cudaMemcpyAsync(tot + 1, uniq + N, sizeof(int), cudaMemcpyDeviceToDevice, st));
  int h[2] = {0, 0};
  SSAMG_CUDA(cudaMemcpyAsync(h, tot, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
  SSAMG_CUDA(cudaStreamSynchronize(st));
  *nr = h[0];
  *nnz = h[1];
  for (void* q : {(void*)cnt, (void*)fill, (void*)perm, (void*)uniq, (void*)flag, (void*)tmp, (void*)tot})
    pool_free(q);
}

void launch_mask_part(double* vals, const int n[3], const int o[3], const PartBoxes& pb,
                      cudaStream_t st) {
  const long long cells = (long long)n[0] * n[1] * n[2];
  const int nb = (int)std::min<long long>(cdiv(cells, NT), 152 * 16);
  k_mask_part<<<nb, NT, 0, st>>>(vals, n[0], n[1], n[2], o[0], o[1], o[2], pb);
  SSAMG_LAUNCH_CHECK();
}

