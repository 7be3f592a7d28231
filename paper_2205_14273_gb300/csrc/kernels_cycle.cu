// V(1,1)-cycle kernels (Section 3.4 relaxation, Eq. relax0; Section 3.2
// restriction R = P^T and prolongation), the FP64 PCG vector kernels
// (Section 4) and the coefficient-gradient kernels of the adjoint solve.
#include <utility>

#include "kernels_common.cuh"

namespace {

constexpr int NT = SSAMG_BLOCK;

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// x = omega M^-1 b (relaxation from a zero guess).
template <class T>
__global__ void k_relax0(int N, const T* dinv, const T* b,
                         T* x) {
  pdl_trigger();
  pdl_wait();
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < N) x[g] = dinv[g] * b[g];
}

// x = omega M^-1 b on blocks [0, nb); row jobs uy = U x on the rest.  The
// diagonal (setup data) is fetched before the wait for the predecessor.
template <class T>
__global__ void __launch_bounds__(NT) k_relax0_u(LevelView<T> L, int nb, const T* b,
                                                 T* x) {
  pdl_trigger();
  if ((int)blockIdx.x < nb) {
    // SSAMG_EW cells per thread, strided by the block: all loads in flight
    const int g0 = blockIdx.x * (NT * SSAMG_EW) + threadIdx.x;
    T d[SSAMG_EW];
#pragma unroll
    for (int m = 0; m < SSAMG_EW; ++m) d[m] = g0 + m * NT < L.N ? L.dinv[g0 + m * NT] : (T)0;
    pdl_wait();
#pragma unroll
    for (int m = 0; m < SSAMG_EW; ++m)
      if (g0 + m * NT < L.N) x[g0 + m * NT] = d[m] * b[g0 + m * NT];
    return;
  }
  u_row_job(
      L, blockIdx.x - nb, [&](int col, int) { return L.dinv[col]; },
      [&](int col, int, T d) { return d * b[col]; });
}

// First pre-relaxation of the cycle straight from the FP64 PCG residual:
// b0 = (T) r, x = omega M^-1 b0 on the cell blocks; uy = U x on the rest.
template <class T>
__global__ void __launch_bounds__(NT) k_relax0_u_first(LevelView<T> L, int nb,
                                                       const double* r64,
                                                       T* b0, T* x) {
  pdl_trigger();
  if ((int)blockIdx.x < nb) {
    const int g0 = blockIdx.x * (NT * SSAMG_EW) + threadIdx.x;
    T d[SSAMG_EW];
#pragma unroll
    for (int m = 0; m < SSAMG_EW; ++m) d[m] = g0 + m * NT < L.N ? L.dinv[g0 + m * NT] : (T)0;
    pdl_wait();
#pragma unroll
    for (int m = 0; m < SSAMG_EW; ++m) {
      const int g = g0 + m * NT;
      if (g < L.N) {
        const T bv = (T)r64[g];
        b0[g] = bv;
        x[g] = d[m] * bv;
      }
    }
    return;
  }
  u_row_job(
      L, blockIdx.x - nb, [&](int col, int) { return L.dinv[col]; },
      [&](int col, int, T d) { return d * (T)r64[col]; });
}

// uy = U x (row jobs only)
template <class T>
__global__ void __launch_bounds__(NT) k_uy(LevelView<T> L, const T* x) {
  pdl_trigger();
  u_row_job(
      L, blockIdx.x, [](int, int) { return 0; }, [&](int col, int, int) { return x[col]; });
}

// r = b - A x
// (with L.nrhs > 1: that many right-hand sides, the blocks of one tile side
// by side, so that the tile's coefficients are read from HBM once)
template <class T, int SH>
__global__ void __launch_bounds__(NT, 4) k_residual(LevelView<T> L, const T* x,
                                                    const T* b, T* r) {
  pdl_trigger();
  __shared__ DPart sp;
  int bid = blockIdx.x, j = 0;
  if (L.nrhs > 1) {
    bid = (int)blockIdx.x / L.nrhs;
    j = (int)blockIdx.x - bid * L.nrhs;
  }
  block_part(L.blk, L.parts, L.np, sp, bid);
  __syncthreads();
  if (j > 0) {
    const long long o = j * L.vstride;
    x += o;
    b += o;
    r += o;
    if (L.uy) L.uy += o;
  }
  pdl_wait();
  if (L.skip && L.skip[sp.prob + j * L.skip_stride].done) return;  // problem already stopped
  TILE_LOOP_AT(c, sp, bid) {
    const int g = sp.off + c;
    r[g] = b[g] - apply_A_sh<SH>(L, sp, x, c);
  }
}

// xo = x + omega M^-1 (b - A x)
// (several right-hand sides per launch as k_residual)
template <class T, int SH>
__global__ void __launch_bounds__(NT, 4) k_relax(LevelView<T> L, const T* x,
                                                 const T* b, T* xo) {
  pdl_trigger();
  __shared__ DPart sp;
  int bid = blockIdx.x, j = 0;
  if (L.nrhs > 1) {
    bid = (int)blockIdx.x / L.nrhs;
    j = (int)blockIdx.x - bid * L.nrhs;
  }
  block_part(L.blk, L.parts, L.np, sp, bid);
  __syncthreads();
  if (j > 0) {
    const long long o = j * L.vstride;
    x += o;
    b += o;
    xo += o;
    if (L.uy) L.uy += o;
  }
  pdl_wait();
  if (L.skip && L.skip[sp.prob + j * L.skip_stride].done) return;  // problem already stopped
  TILE_LOOP_AT(c, sp, bid) {
    const int g = sp.off + c;
    xo[g] = fma(L.dinv[g], b[g] - apply_A_sh<SH>(L, sp, x, c), x[g]);
  }
}

// r = b - A x and xo = x + omega M^-1 (b - A x) for R right-hand sides per
// thread (shapes with every entry per cell): the coefficients of a cell are
// loaded once for all of them.  Right-hand side q's vectors (and U x) lie
// q L.vstride elements after the first's, its scalars q L.skip_stride after
// the first's; a right-hand side whose problem has stopped is not written.
// (blocks per SM, measured on the batched workload's levels with four
// right-hand sides: the fixed shapes run best with 64 registers, 4 blocks;
// the general shape's per-part dispatch with 48, 5 blocks, although it then
// spills a few words: 729 vs 921 us on a 15-point level of 18M cells)
template <class T, int SH>
constexpr int rhs_min_blocks() {
  return (SH == SH_UGEN && sizeof(T) == 4) ? 5 : 4;
}
template <class T, int SH, int R, bool RELAX>
__global__ void __launch_bounds__(NT, rhs_min_blocks<T, SH>()) k_cycle_r(LevelView<T> L, const T* x, const T* b,
                                                   T* out) {
  pdl_trigger();
  __shared__ DPart sp;
  block_part(L.blk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  const long long vs = L.vstride;
  unsigned act = 0;
#pragma unroll
  for (int q = 0; q < R; ++q)
    if (!L.skip || !L.skip[sp.prob + q * L.skip_stride].done) act |= 1u << q;
  if (!act) return;  // every right-hand side of the problem stopped
  TILE_LOOP(c, sp) {
    const int g = sp.off + c;
    T acc[R];
    apply_A_sh_r<SH, R>(L, sp, x, c, vs, acc);
    const T dv = RELAX ? L.dinv[g] : (T)0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      if (!((act >> q) & 1u)) continue;
      const long long o = g + q * vs;
      if (RELAX)
        out[o] = fma(dv, b[o] - acc[q], x[o]);
      else
        out[o] = b[o] - acc[q];
    }
  }
}

// Last post-relaxation of the cycle: t = x + omega M^-1 (b - A x) written as
// the FP64 preconditioned residual z, with the block partials of r.z and
// r.zprev (flexible CG; zprev then takes z) for the PCG's beta.
template <class T, int SH>
__global__ void __launch_bounds__(NT, 4) k_relax_final(LevelView<T> L, const T* x,
                                                       const T* b,
                                                       double* z,
                                                       const double* rpcg,
                                                       double* zprev, int flex,
                                                       double* partial) {
  pdl_trigger();
  __shared__ DPart sp;
  __shared__ double sh[NT];
  block_part(L.blk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  if (L.skip && L.skip[sp.prob].done) return;  // problem already stopped
  double s0 = 0.0, s1 = 0.0;
  TILE_LOOP(c, sp) {
    const int g = sp.off + c;
    // the FP64 operands are fetched with the stencil's, not after it (zprev
    // is a valid buffer even without flexible CG: z itself, read before its
    // store and then unused)
    const double rv = rpcg[g];
    const double zo = zprev[g];
    const double zv = (double)fma(L.dinv[g], b[g] - apply_A_sh<SH>(L, sp, x, c), x[g]);
    z[g] = zv;
    s0 = fma(rv, zv, s0);
    if (flex) {
      s1 = fma(rv, zo, s1);
      zprev[g] = zv;
    }
  }
  const double t0 = block_sum<NT>(s0, sh);
  const double t1 = block_sum<NT>(s1, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = t0;
    partial[2 * blockIdx.x + 1] = t1;
  }
}

// ---------------------------------------------------------------------------
// Checked 7-point operator applies over bricks (levels of shape SH_K7: entries
// [C, -x, +x, -y, +y, -z, +z], some of them constant per part).  A block takes
// an SSAMG_BRICK_X x _Y x _Z brick of one part and each thread marches one
// (i, j) column along z, carrying x at k-1 and k in registers: no cell
// coordinate needs a division, and each x value comes from DRAM once (the
// in-plane neighbours hit L1).  The operation Op supplies the per-cell inputs
// of its epilogue (`load`, issued ahead of the stencil's loads, so that a
// cell costs one memory round trip) and the epilogue (`apply`).  The stencil
// terms are summed in the order of stencil7_canon_checked, so a cell's A x is
// bitwise that of the cell-tile kernels.
// ---------------------------------------------------------------------------
template <class T, int KM, class Op>
__device__ __forceinline__ void brick7(const LevelView<T>& L, const DPart& sp, const T* x,
                                       Op& op) {
  const int bl = (int)blockIdx.x - sp.bblk0;
  const int bx = bl % sp.bb[0];
  const int byz = bl / sp.bb[0];
  const int by = byz % sp.bb[1];
  const int bz = byz / sp.bb[1];
  const int nx = sp.n[0], ny = sp.n[1], nz = sp.n[2], nxy = nx * ny;
  const int i = bx * SSAMG_BRICK_X + (int)threadIdx.x % SSAMG_BRICK_X;
  const int j = by * SSAMG_BRICK_Y + (int)threadIdx.x / SSAMG_BRICK_X;
  if (i >= nx || j >= ny) return;
  const int k0 = bz * SSAMG_BRICK_Z;
  const int kend = min(k0 + SSAMG_BRICK_Z, nz);
  const unsigned vm = sp.varmask;
  const T* xp0 = x + sp.off;
  const bool bw = i > 0, be = i < nx - 1, bs = j > 0, bn = j < ny - 1;
  const bool face_ij = !(bw && be && bs && bn);
  const T c1 = const_of<T>(sp, 1), c2 = const_of<T>(sp, 2), c3 = const_of<T>(sp, 3),
          c4 = const_of<T>(sp, 4), c5 = const_of<T>(sp, 5), c6 = const_of<T>(sp, 6),
          c0 = const_of<T>(sp, 0);
  int c = (k0 * ny + j) * nx + i;
  T xm = k0 > 0 ? xp0[c - nxy] : (T)0;
  T xcur = xp0[c];
  T xz = k0 + 1 < nz ? xp0[c + nxy] : (T)0;
  auto in = op.load(sp.off + c);
  // KM 0: all entries constant; 1: only the diagonal may vary per cell; 2: any
  const bool dvar = KM >= 1 && (vm & 1u);
  T d0 = dvar ? L.coef[sp.coef[0] + c] : c0;
#pragma unroll 1
  for (int k = k0; k < kend; ++k, c += nxy) {
    // the next cell's streamed inputs (x two planes up, the epilogue's
    // inputs) are requested before this cell's arithmetic, so that two
    // cells' DRAM loads are in flight per thread
    const bool more = k + 1 < kend;
    const T xz2 = more && k + 2 < nz ? xp0[c + 2 * nxy] : (T)0;
    const auto in2 = more ? op.load(sp.off + c + nxy) : in;
    const T d2 = dvar && more ? L.coef[sp.coef[0] + c + nxy] : d0;
    const T xw = bw ? xp0[c - 1] : (T)0;
    const T xe = be ? xp0[c + 1] : (T)0;
    const T xs = bs ? xp0[c - nx] : (T)0;
    const T xn = bn ? xp0[c + nx] : (T)0;
    const T a0 = d0;
    const T a1 = (KM == 2 && (vm & 2u)) ? L.coef[sp.coef[1] + c] : c1;
    const T a2 = (KM == 2 && (vm & 4u)) ? L.coef[sp.coef[2] + c] : c2;
    const T a3 = (KM == 2 && (vm & 8u)) ? L.coef[sp.coef[3] + c] : c3;
    const T a4 = (KM == 2 && (vm & 16u)) ? L.coef[sp.coef[4] + c] : c4;
    const T a5 = (KM == 2 && (vm & 32u)) ? L.coef[sp.coef[5] + c] : c5;
    const T a6 = (KM == 2 && (vm & 64u)) ? L.coef[sp.coef[6] + c] : c6;
    T acc = (T)0;
    acc = fma(a0, xcur, acc);
    acc = fma(a1, xw, acc);
    acc = fma(a2, xe, acc);
    acc = fma(a3, xs, acc);
    acc = fma(a4, xn, acc);
    acc = fma(a5, k > 0 ? xm : (T)0, acc);
    acc = fma(a6, xz, acc);
    if (sp.has_u && (sp.has_u > 1 || face_ij || k == 0 || k == nz - 1)) acc += L.uy[sp.off + c];
    op.apply(sp.off + c, acc, xcur, in);
    xm = xcur;
    xcur = xz;
    xz = xz2;
    in = in2;
    d0 = d2;
  }
}

// The instance of a brick kernel for a level's coefficient mode (Level::kvar).
template <class F>
F pick_km(int km, F f0, F f1, F f2) {
  return km == 0 ? f0 : km == 1 ? f1 : f2;
}

// Resident blocks per SM the brick residual and relaxation are compiled for:
// as many as fit without register spills.
template <class T, int KM>
constexpr int brick_min_blocks() {
  return sizeof(T) == 8 ? (KM == 2 ? 4 : 5) : (KM == 2 ? 5 : 6);
}

template <class T>
struct ResidualOp {
  const T* b;
  T* r;
  __device__ T load(int g) const { return b[g]; }
  __device__ void apply(int g, T ax, T, T bv) const { r[g] = bv - ax; }
};

template <class T>
struct RelaxOp {
  const T* b;
  const T* dinv;
  T* xo;
  struct In {
    T b, d;
  };
  __device__ In load(int g) const { return In{b[g], dinv[g]}; }
  __device__ void apply(int g, T ax, T xg, In in) const { xo[g] = fma(in.d, in.b - ax, xg); }
};

struct PcgInitOp {
  const double* b;
  double* r;
  double bb, rr;
  __device__ double load(int g) const { return b[g]; }
  __device__ void apply(int g, double ax, double, double bv) {
    const double rv = bv - ax;
    r[g] = rv;
    bb = fma(bv, bv, bb);
    rr = fma(rv, rv, rr);
  }
};

struct SpmvDotOp {
  double* q;
  double s;
  __device__ int load(int) const { return 0; }
  __device__ void apply(int g, double ax, double pg, int) {
    q[g] = ax;
    s = fma(pg, ax, s);
  }
};

// The cycle's last post-relaxation as the PCG runs it (see k_relax_final).
template <class T>
struct RelaxFinalOp {
  const T* b;
  const T* dinv;
  double* z;
  const double* rpcg;
  double* zprev;
  int flex;
  double s0, s1;
  struct In {
    T b, d;
    double r, zo;
  };
  __device__ In load(int g) const { return In{b[g], dinv[g], rpcg[g], zprev[g]}; }
  __device__ void apply(int g, T ax, T xg, In in) {
    const double zv = (double)fma(in.d, in.b - ax, xg);
    z[g] = zv;
    s0 = fma(in.r, zv, s0);
    if (flex) {
      s1 = fma(in.r, in.zo, s1);
      zprev[g] = zv;
    }
  }
};

template <class T, int KM>
__global__ void __launch_bounds__(NT, brick_min_blocks<T, KM>()) k7b_residual(LevelView<T> L, const T* x, const T* b, T* r) {
  pdl_trigger();
  __shared__ DPart sp;
  block_part(L.bblk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  if (L.skip && L.skip[sp.prob].done) return;  // problem already stopped
  ResidualOp<T> op{b, r};
  brick7<T, KM>(L, sp, x, op);
}

template <class T, int KM>
__global__ void __launch_bounds__(NT, brick_min_blocks<T, KM>()) k7b_relax(LevelView<T> L, const T* x, const T* b, T* xo) {
  pdl_trigger();
  __shared__ DPart sp;
  block_part(L.bblk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  if (L.skip && L.skip[sp.prob].done) return;  // problem already stopped
  RelaxOp<T> op{b, L.dinv, xo};
  brick7<T, KM>(L, sp, x, op);
}

template <class T, int KM>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 5 : 4) k7b_relax_final(LevelView<T> L, const T* x, const T* b,
                                                      double* z, const double* rpcg,
                                                      double* zprev, int flex, double* partial) {
  pdl_trigger();
  __shared__ DPart sp;
  __shared__ double sh[NT];
  block_part(L.bblk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  if (L.skip && L.skip[sp.prob].done) return;  // problem already stopped
  RelaxFinalOp<T> op{b, L.dinv, z, rpcg, zprev, flex, 0.0, 0.0};
  brick7<T, KM>(L, sp, x, op);
  const double t0 = block_sum<NT>(op.s0, sh);
  const double t1 = block_sum<NT>(op.s1, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = t0;
    partial[2 * blockIdx.x + 1] = t1;
  }
}

template <int KM>
__global__ void __launch_bounds__(NT, 4) k7b_pcg_init(LevelView<double> L, const double* b,
                                                   const double* x, double* r, double* partial) {
  pdl_trigger();
  __shared__ DPart sp;
  __shared__ double sh[NT];
  block_part(L.bblk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  PcgInitOp op{b, r, 0.0, 0.0};
  brick7<double, KM>(L, sp, x, op);
  const double s0 = block_sum<NT>(op.bb, sh);
  const double s1 = block_sum<NT>(op.rr, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0;
    partial[2 * blockIdx.x + 1] = s1;
  }
}

template <int KM>
__global__ void __launch_bounds__(NT, 4) k7b_spmv_dot(LevelView<double> L, const double* p, double* q,
                                                   double* partial) {
  pdl_trigger();
  __shared__ DPart sp;
  __shared__ double sh[NT];
  block_part(L.bblk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  if (L.skip && L.skip[sp.prob].done) return;  // problem already stopped
  SpmvDotOp op{q, 0.0};
  brick7<double, KM>(L, sp, p, op);
  const double t = block_sum<NT>(op.s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// Restriction row of a coupling column (fine cells, side weights) and the
// column's omega M^-1 (setup data of a row job entry).
template <class T>
struct RCol {
  int j0, j1, j2;
  T w1, w2, d;
};

// bc = P^T r, one coarse cell per thread: the anchor (weight 1) and the two
// fine points beside it along d* (weights PE of the west one, PW of the east).
template <class T>
__global__ void __launch_bounds__(NT) k_restrict(LevelView<T> F, LevelView<T> C,
                                                 const T* r, T* bc, T* xc, int nb) {
  pdl_trigger();
  __shared__ DPart fp;
  __shared__ DPart cp;
  if ((int)blockIdx.x >= nb) {
    // row jobs of the coarse level's pre-relaxation: uy = U x with
    // x = omega M^-1 b at each coupling's column, b rebuilt there from the
    // column's restriction row exactly as the tiles compute it
    u_row_job(
        C, blockIdx.x - nb,
        [&](int col, int q) {
          return RCol<T>{C.u_rj[3 * q], C.u_rj[3 * q + 1], C.u_rj[3 * q + 2], C.u_rw[2 * q],
                         C.u_rw[2 * q + 1], C.dinv[col]};
        },
        [&](int, int, const RCol<T>& rc) {
          T v = r[rc.j0];
          if (rc.j1 >= 0) v = fma(rc.w1, r[rc.j1], v);
          if (rc.j2 >= 0) v = fma(rc.w2, r[rc.j2], v);
          return rc.d * v;
        });
    return;
  }
  int p = block_part(C.blk, C.parts, C.np, cp);
  part_of(F.parts, p, fp);
  __syncthreads();
  pdl_wait();
  if (C.skip && C.skip[cp.prob].done) return;  // problem already stopped
  TILE_LOOP_UNROLLED(cc, cp) {
    int I[3];
    cell_coords(cp, cc, I[0], I[1], I[2]);
    const int d = fp.dstar;
    T v;
    if (d < 0) {
      v = r[fp.off + (I[2] * fp.n[1] + I[1]) * fp.n[0] + I[0]];
    } else {
      int f[3] = {I[0], I[1], I[2]};
      const int anchor = 2 * I[d] + fp.par;
      f[d] = anchor;
      const int sd = (d == 0) ? 1 : (d == 1 ? fp.n[0] : fp.n[0] * fp.n[1]);
      const int fa = fp.off + (f[2] * fp.n[1] + f[1]) * fp.n[0] + f[0];
      v = r[fa];
      if (anchor - 1 >= 0) {
        f[d] = anchor - 1;
        v = fma(F.Pe[fp.poff + fine_point_index(fp, f[0], f[1], f[2])], r[fa - sd], v);
      }
      if (anchor + 1 < fp.n[d]) {
        f[d] = anchor + 1;
        v = fma(F.Pw[fp.poff + fine_point_index(fp, f[0], f[1], f[2])], r[fa + sd], v);
      }
    }
    bc[cp.off + cc] = v;
    if (xc) xc[cp.off + cc] = C.dinv[cp.off + cc] * v;  // pre-relaxation from zero
  }
}

// Coarse-side P row of a coupling column (setup data of a row job entry).
template <class T>
struct PCol {
  int j0, j1;
  T w0, w1;
};

// ---------------------------------------------------------------------------
// Restriction and prolongation over bricks.  On levels whose bricks are well
// filled, a block takes a 32 x 8 x 8 brick of one part and each thread walks
// one (i, j) column along z.  The code is specialised per coarsening
// direction D of the part (block-uniform): the row of P (or of P^T) of a
// cell follows from the column's fixed coordinates and k by running index
// updates, not from a division per cell.  A column's setup data (P weights,
// smoother diagonal) is fetched before the wait for the predecessor and the
// vectors of all its cells are requested before any of them is combined.
// Each cell's result is computed in the same operation order as the
// cell-tile kernels above, so the two forms agree bit for bit.
// ---------------------------------------------------------------------------
constexpr int RP_Z = SSAMG_BRICK_Z;

// The thread's column (i, j) and first z of its brick; false when the column
// lies outside the part.  The brick's position comes from shared memory,
// decoded once per block (bpos[0..2], written by thread 0 of the block).
__device__ __forceinline__ void rp_brick_origin(const DPart& sp, int* bpos) {
  if (threadIdx.x == 0) {
    const int bl = (int)blockIdx.x - sp.bblk0;
    bpos[0] = bl % sp.bb[0];
    const int byz = bl / sp.bb[0];
    bpos[1] = byz % sp.bb[1];
    bpos[2] = byz / sp.bb[1];
  }
}
__device__ __forceinline__ bool rp_column(const DPart& sp, const int* bpos, int& i, int& j,
                                          int& k0) {
  i = bpos[0] * SSAMG_BRICK_X + (int)threadIdx.x % SSAMG_BRICK_X;
  j = bpos[1] * SSAMG_BRICK_Y + (int)threadIdx.x / SSAMG_BRICK_X;
  k0 = bpos[2] * SSAMG_BRICK_Z;
  return i < sp.n[0] && j < sp.n[1];
}

// Restriction of one column of coarse cells (I0, I1, K0 ..), part coarsened
// along D (-1: not coarsened).  Side weights and the diagonal are fetched
// before pdl_wait(); then the residuals of every cell, then the sums.
template <int D, class T>
__device__ __forceinline__ void restrict_column(const LevelView<T>& F, const LevelView<T>& C,
                                                const DPart& fp, const DPart& cp, int I0, int I1,
                                                int K0, int kend, const T* r, T* bc, T* xc) {
  const int n0 = fp.n[0], n1 = fp.n[1], nxy = n0 * n1;
  const int sd = D == 0 ? 1 : D == 1 ? n0 : nxy;
  // fine anchor of the first cell and its step per coarse k
  const int a0 = D == 0 ? 2 * I0 + fp.par : I0;
  const int a1 = D == 1 ? 2 * I1 + fp.par : I1;
  int fa = fp.off + ((D == 2 ? 2 * K0 + fp.par : K0) * n1 + a1) * n0 + a0;
  const int dfa = D == 2 ? 2 * nxy : nxy;
  // fine-point (P array) index of the west side's fine point, its step, and
  // the east side's offset from it
  const int nf0 = fp.nf[0], nf1 = fp.nf[1], nfxy = nf0 * nf1;
  int pw = 0, dpw = 0, pe_off = 0;
  if (D == 0) {
    pw = fp.poff + (K0 * nf1 + I1) * nf0 + ((a0 - 1 + fp.par) >> 1);
    dpw = nfxy;
    pe_off = 1;
  } else if (D == 1) {
    pw = fp.poff + (K0 * nf1 + ((a1 - 1 + fp.par) >> 1)) * nf0 + I0;
    dpw = nfxy;
    pe_off = nf0;
  } else if (D == 2) {
    pw = fp.poff + (((2 * K0 + fp.par - 1 + fp.par) >> 1) * nf1 + I1) * nf0 + I0;
    dpw = nfxy;
    pe_off = nfxy;
  }
  const int ad = D == 0 ? a0 : D == 1 ? a1 : 0;
  const int nd = D == 0 ? n0 : D == 1 ? n1 : fp.n[2];
  T w1[RP_Z], w2[RP_Z], dv[RP_Z];
  bool hw[RP_Z], he[RP_Z];
  int cc0 = cp.off + (K0 * cp.n[1] + I1) * cp.n[0] + I0;
  const int dcc = cp.n[0] * cp.n[1];
#pragma unroll
  for (int t = 0; t < RP_Z; ++t) {
    const bool in = K0 + t < kend;
    const int anc = D == 2 ? 2 * (K0 + t) + fp.par : ad;
    hw[t] = D >= 0 && in && anc - 1 >= 0;
    he[t] = D >= 0 && in && anc + 1 < nd;
    w1[t] = hw[t] ? F.Pe[pw + t * dpw] : (T)0;
    w2[t] = he[t] ? F.Pw[pw + t * dpw + pe_off] : (T)0;
    dv[t] = (xc && in) ? C.dinv[cc0 + t * dcc] : (T)0;
  }
  pdl_wait();
  if (C.skip && C.skip[cp.prob].done) return;  // problem already stopped
  T r0[RP_Z], r1[RP_Z], r2[RP_Z];
#pragma unroll
  for (int t = 0; t < RP_Z; ++t) {
    const bool in = K0 + t < kend;
    const int f = fa + t * dfa;
    r0[t] = in ? r[f] : (T)0;
    r1[t] = hw[t] ? r[f - sd] : (T)0;
    r2[t] = he[t] ? r[f + sd] : (T)0;
  }
#pragma unroll
  for (int t = 0; t < RP_Z; ++t) {
    if (K0 + t >= kend) break;
    T v = r0[t];
    if (hw[t]) v = fma(w1[t], r1[t], v);
    if (he[t]) v = fma(w2[t], r2[t], v);
    bc[cc0 + t * dcc] = v;
    if (xc) xc[cc0 + t * dcc] = dv[t] * v;  // pre-relaxation from zero
  }
}

template <class T>
__global__ void __launch_bounds__(NT) k_restrict_b(LevelView<T> F, LevelView<T> C, const T* r,
                                                   T* bc, T* xc, int nb) {
  pdl_trigger();
  __shared__ DPart fp;
  __shared__ DPart cp;
  __shared__ int bpos[3];
  if ((int)blockIdx.x >= nb) {
    u_row_job(
        C, blockIdx.x - nb,
        [&](int col, int q) {
          return RCol<T>{C.u_rj[3 * q], C.u_rj[3 * q + 1], C.u_rj[3 * q + 2], C.u_rw[2 * q],
                         C.u_rw[2 * q + 1], C.dinv[col]};
        },
        [&](int, int, const RCol<T>& rc) {
          T v = r[rc.j0];
          if (rc.j1 >= 0) v = fma(rc.w1, r[rc.j1], v);
          if (rc.j2 >= 0) v = fma(rc.w2, r[rc.j2], v);
          return rc.d * v;
        });
    return;
  }
  const int p = block_part(C.bblk, C.parts, C.np, cp);
  part_of(F.parts, p, fp);
  __syncthreads();
  rp_brick_origin(cp, bpos);
  __syncthreads();
  int I0, I1, K0;
  const bool ok = rp_column(cp, bpos, I0, I1, K0);
  const int kend = min(K0 + RP_Z, cp.n[2]);
  if (!ok) {
    pdl_wait();
    return;
  }
  switch (fp.dstar) {
    case 0: restrict_column<0>(F, C, fp, cp, I0, I1, K0, kend, r, bc, xc); break;
    case 1: restrict_column<1>(F, C, fp, cp, I0, I1, K0, kend, r, bc, xc); break;
    case 2: restrict_column<2>(F, C, fp, cp, I0, I1, K0, kend, r, bc, xc); break;
    default: restrict_column<-1>(F, C, fp, cp, I0, I1, K0, kend, r, bc, xc); break;
  }
}

// Prolongation x_out = x_in + P e of one column of PZ fine cells
// (i, j, k0 ..), part coarsened along D (-1: not coarsened, P = I).  The
// prolongation walks half bricks (PZ = RP_Z / 2): fewer registers per
// thread, twice the blocks, measured faster than whole bricks.
constexpr int PZ = RP_Z / 2;
template <int D, class T>
__device__ __forceinline__ void prolong_column(const LevelView<T>& F, const DPart& fp, int i,
                                               int j, int k0, int kend, const T* ec,
                                               const T* xin, T* xout) {
  const int n0 = fp.n[0], n1 = fp.n[1], nxy = n0 * n1;
  const int cn0 = fp.cn[0], cn1 = fp.cn[1], cnxy = cn0 * cn1;
  const int nf0 = fp.nf[0], nf1 = fp.nf[1], nfxy = nf0 * nf1;
  const int par = fp.par;
  // per cell: up to two coarse columns and their weights, in p_row's order
  int j0[PZ], j1[PZ];
  T w0[PZ], w1[PZ];
#pragma unroll
  for (int t = 0; t < PZ; ++t) {
    const int k = k0 + t;
    j0[t] = j1[t] = -1;
    w0[t] = w1[t] = (T)0;
    if (k >= kend) continue;
    if (D < 0) {
      j0[t] = fp.coff + (k * cn1 + j) * cn0 + i;
      w0[t] = (T)1;
      continue;
    }
    const int cd = D == 0 ? i : D == 1 ? j : k;
    const int nd = D == 0 ? n0 : D == 1 ? n1 : fp.n[2];
    // coarse index with the D coordinate replaced by v
    auto at = [&](int v) {
      return fp.coff + ((D == 2 ? v : k) * cn1 + (D == 1 ? v : j)) * cn0 + (D == 0 ? v : i);
    };
    if (((cd + par) & 1) == 0) {
      j0[t] = at((cd - par) >> 1);
      w0[t] = (T)1;
      continue;
    }
    const int Fi = fp.poff + ((D == 2 ? (k + par) >> 1 : k) * nf1 + (D == 1 ? (j + par) >> 1 : j)) * nf0 +
                   (D == 0 ? (i + par) >> 1 : i);
    if (cd - 1 >= 0) {
      j0[t] = at((cd - 1 - par) >> 1);
      w0[t] = F.Pw[Fi];
    }
    if (cd + 1 < nd) {
      j1[t] = at((cd + 1 - par) >> 1);
      w1[t] = F.Pe[Fi];
    }
    if (j0[t] < 0) {  // only the east neighbour: keep it first
      j0[t] = j1[t];
      w0[t] = w1[t];
      j1[t] = -1;
      w1[t] = (T)0;
    }
  }
  (void)cnxy;
  (void)nfxy;
  pdl_wait();
  if (F.skip && F.skip[fp.prob].done) return;  // problem already stopped
  const int c0 = fp.off + (k0 * n1 + j) * n0 + i;
  T xv[PZ], e0[PZ], e1[PZ];
#pragma unroll
  for (int t = 0; t < PZ; ++t) {
    const bool in = k0 + t < kend;
    xv[t] = in ? xin[c0 + t * nxy] : (T)0;
    e0[t] = in && j0[t] >= 0 ? ec[j0[t]] : (T)0;
    e1[t] = in && j1[t] >= 0 ? ec[j1[t]] : (T)0;
  }
#pragma unroll
  for (int t = 0; t < PZ; ++t) {
    if (k0 + t >= kend) break;
    T v = xv[t];
    if (j0[t] >= 0) v = fma(w0[t], e0[t], v);
    if (j1[t] >= 0) v = fma(w1[t], e1[t], v);
    xout[c0 + t * nxy] = v;
  }
}

template <class T>
__global__ void __launch_bounds__(NT) k_prolong_ub(LevelView<T> F, const T* ec, const T* xin,
                                                   T* xout, int nb) {
  pdl_trigger();
  __shared__ DPart fp;
  __shared__ int bpos[3];
  if ((int)blockIdx.x >= nb) {
    u_row_job(
        F, blockIdx.x - nb,
        [&](int, int q) {
          return PCol<T>{F.u_pj[2 * q], F.u_pj[2 * q + 1], F.u_pw[2 * q], F.u_pw[2 * q + 1]};
        },
        [&](int col, int, const PCol<T>& pc) {
          T v = xin[col];
          if (pc.j0 >= 0) v = fma(pc.w0, ec[pc.j0], v);
          if (pc.j1 >= 0) v = fma(pc.w1, ec[pc.j1], v);
          return v;
        });
    return;
  }
  // two blocks per brick: block b takes the half (b & 1) of brick b >> 1
  block_part(F.bblk, F.parts, F.np, fp, (int)blockIdx.x >> 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int bl = ((int)blockIdx.x >> 1) - fp.bblk0;
    bpos[0] = bl % fp.bb[0];
    const int byz = bl / fp.bb[0];
    bpos[1] = byz % fp.bb[1];
    bpos[2] = byz / fp.bb[1];
  }
  __syncthreads();
  int i, j, k0;
  const bool ok = rp_column(fp, bpos, i, j, k0);
  k0 += ((int)blockIdx.x & 1) * PZ;
  const int kend = min(k0 + PZ, fp.n[2]);
  if (!ok) {
    pdl_wait();
    return;
  }
  switch (fp.dstar) {
    case 0: prolong_column<0>(F, fp, i, j, k0, kend, ec, xin, xout); break;
    case 1: prolong_column<1>(F, fp, i, j, k0, kend, ec, xin, xout); break;
    case 2: prolong_column<2>(F, fp, i, j, k0, kend, ec, xin, xout); break;
    default: prolong_column<-1>(F, fp, i, j, k0, kend, ec, xin, xout); break;
  }
}


// xout = xin + P ec on the cell tiles; row jobs uy = U xout, where xout at a
// coupling's column is rebuilt from xin and the column's P row (precomputed
// at setup), so the two roles need no ordering.  P rows are setup data and
// are fetched before the wait for the predecessor.
template <class T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 8 : 6) k_prolong_u(LevelView<T> F, const T* ec,
                                                  const T* xin, T* xout,
                                                  int nb) {
  pdl_trigger();
  __shared__ DPart fp;
  if ((int)blockIdx.x >= nb) {
    u_row_job(
        F, blockIdx.x - nb,
        [&](int, int q) {
          return PCol<T>{F.u_pj[2 * q], F.u_pj[2 * q + 1], F.u_pw[2 * q], F.u_pw[2 * q + 1]};
        },
        [&](int col, int, const PCol<T>& pc) {
          T v = xin[col];
          if (pc.j0 >= 0) v = fma(pc.w0, ec[pc.j0], v);
          if (pc.j1 >= 0) v = fma(pc.w1, ec[pc.j1], v);
          return v;
        });
    return;
  }
  int p = block_part(F.blk, F.parts, F.np, fp);
  __syncthreads();
  // the first tile cell's P row (setup data) is fetched before the wait
  const int cfirst = ((int)blockIdx.x - fp.blk0) * fp.cpt * SSAMG_BLOCK + (int)threadIdx.x;
  PRow<T> pr0{-1, -1, (T)0, (T)0};
  if (cfirst < fp.ncell) {
    int i, j, k;
    cell_coords(fp, cfirst, i, j, k);
    pr0 = p_row(fp, F.Pw, F.Pe, i, j, k);
  }
  pdl_wait();
  if (F.skip && F.skip[fp.prob].done) return;  // problem already stopped
  TILE_LOOP_UNROLLED(c, fp) {
    PRow<T> pr = pr0;
    if (c != cfirst) {
      int i, j, k;
      cell_coords(fp, c, i, j, k);
      pr = p_row(fp, F.Pw, F.Pe, i, j, k);
    }
    xout[fp.off + c] = add_p_row(xin[fp.off + c], pr, ec);
  }
  (void)p;
}

// x += P ec, one fine cell per thread.
template <class T>
__global__ void __launch_bounds__(NT) k_prolong(LevelView<T> F, const T* ec,
                                                T* x) {
  pdl_trigger();
  __shared__ DPart fp;
  int p = block_part(F.blk, F.parts, F.np, fp);
  __syncthreads();
  pdl_wait();
  TILE_LOOP(c, fp) {
    int i, j, k;
    cell_coords(fp, c, i, j, k);
    x[fp.off + c] = add_p_row(x[fp.off + c], p_row(fp, F.Pw, F.Pe, i, j, k), ec);
  }
}

// Coarsest level: x = (L L^T)^-1 b in FP64 with one warp; small factors are
// staged in shared memory first (one coalesced load instead of a dependent
// global load per row).
template <class T>
__global__ void k_coarse_solve(int n, const double* Lg, const T* b,
                               T* x, int staged) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ double sm[];
  double* y = sm;
  const double* Lf = Lg;
  const int l = threadIdx.x;
  if (staged) {
    double* Ls = sm + n;
    for (int t = l; t < n * n; t += 32) Ls[t] = Lg[t];
    __syncwarp();
    Lf = Ls;
  }
  for (int i = 0; i < n; ++i) {
    const double* ri = Lf + (long long)i * n;
    double s = 0.0;
    for (int k = l; k < i; k += 32) s += ri[k] * y[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) y[i] = ((double)b[i] - s) / ri[i];
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = 0.0;
    for (int k = i + 1 + l; k < n; k += 32) s += Lf[(long long)k * n + i] * y[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (l == 0) y[i] = (y[i] - s) / Lf[(long long)i * n + i];
    __syncwarp();
  }
  for (int i = l; i < n; i += 32) x[i] = (T)y[i];
}

// ---------------------------------------------------------------------------
// Fused coarse tail: every small level of the V-cycle in one cooperative
// launch.  The steps are those of the per-level kernels above (pre-relaxation
// with U x, residual, restriction, coarsest solve, prolongation with U x,
// post-relaxation); a grid barrier separates them instead of a kernel
// boundary.  Every thread handles at most a few cells or coupling rows per
// step, so a step costs one or two dependent memory round trips.
// ---------------------------------------------------------------------------
constexpr int TB = SSAMG_TAIL_BLOCK;

// Grid barrier over gridDim.x co-resident blocks (cooperative launch).  Each
// block's thread 0 adds to one counter with release semantics; block 0 adds
// 2^31 - (nblocks - 1 + gb->extra), the others 1, so the counter's top bit
// flips exactly when every block (and gb->extra further arrivals, 0 outside
// the self-test) has arrived.  Waiters poll with acquire semantics (which
// also makes the other blocks' writes visible through this SM's L1).  The
// wait is bounded: after gb->cap polls the block records the failure in
// gb->err and continues, and the caller reports a timeout.
__device__ __forceinline__ void grid_barrier(TailBarrier* gb) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* ctr = &gb->count;
    const unsigned cap = *(volatile unsigned*)&gb->cap;
    const unsigned extra = (unsigned)*(volatile int*)&gb->extra;
    const unsigned nb = (blockIdx.x == 0) ? 0x80000000u - (gridDim.x - 1u + extra) : 1u;
    unsigned old, cur;
    asm volatile("atom.add.release.gpu.u32 %0,[%1],%2;" : "=r"(old) : "l"(ctr), "r"(nb) : "memory");
    unsigned spins = 0;
    for (;;) {
      asm volatile("ld.acquire.gpu.u32 %0,[%1];" : "=r"(cur) : "l"(ctr) : "memory");
      if ((old ^ cur) & 0x80000000u) break;
      if (++spins > cap) {
        atomicExch(&gb->err, 1);
        break;
      }
      __nanosleep(32);
    }
  }
  __syncthreads();
}

// Self-test kernel: every block meets at one grid barrier.
__global__ void k_barrier_selftest(TailBarrier* gb) { grid_barrier(gb); }

// Operator apply of a tail level with the level's stencil shape (the same
// specialised, unchecked stencils as the per-level kernels).
template <class T>
__device__ __forceinline__ T tail_apply(const LevelView<T>& L, const DPart& sp,
                                        const T* __restrict__ x, int c, int shape) {
  switch (shape) {
    case SH_U7: return apply_A_sh<SH_U7>(L, sp, x, c);
    case SH_U15: return apply_A_sh<SH_U15>(L, sp, x, c);
    case SH_C27: return apply_A_sh<SH_C27>(L, sp, x, c);
    case SH_UGEN: return apply_A_sh<SH_UGEN>(L, sp, x, c);
    case SH_K7: return apply_A_sh<SH_K7>(L, sp, x, c);
    default: return apply_A_sh<SH_CHECKED>(L, sp, x, c);
  }
}

__device__ __forceinline__ int tail_part(const int* __restrict__ cs, int np, int g) {
  int p = 0;
  while (p + 1 < np && __ldg(cs + p + 1) <= g) ++p;
  return p;
}

// ONE = true: a single CTA of SSAMG_TAIL_CTA threads runs the tail, with
// __syncthreads() as the step barrier and the level table staged in shared
// memory (launched like the other cycle kernels, with programmatic dependent
// launch).  ONE = false: a cooperative grid with grid_barrier().
template <class T, bool ONE>
__global__ void __launch_bounds__(ONE ? SSAMG_TAIL_CTA : TB)
    k_vtail(const TailLevel<T>* lvg, int nlev, const double* cinv,
            int nL, int coarse_direct, TailBarrier* gb) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const TailLevel<T>* lv = lvg;
  if constexpr (ONE) {
    // shared memory: the level table, then every level's part descriptors
    // (the table's part pointers are redirected there)
    pdl_trigger();
    extern __shared__ __align__(16) int tail_smem[];
    TailLevel<T>* slv = reinterpret_cast<TailLevel<T>*>(tail_smem);
    const int nw = nlev * (int)(sizeof(TailLevel<T>) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(lvg);
    for (int t = threadIdx.x; t < nw; t += blockDim.x) tail_smem[t] = __ldg(src + t);
    __syncthreads();
    DPart* sparts = reinterpret_cast<DPart*>(slv + nlev);
    constexpr int dw = (int)(sizeof(DPart) / sizeof(int));
    for (int l = 0; l < nlev; ++l) {
      const int* ps = reinterpret_cast<const int*>(slv[l].L.parts);
      int* pd = reinterpret_cast<int*>(sparts);
      const int n = slv[l].L.np * dw;
      for (int t = threadIdx.x; t < n; t += blockDim.x) pd[t] = __ldg(ps + t);
      __syncthreads();
      if (threadIdx.x == 0) slv[l].L.parts = sparts;
      sparts += slv[l].L.np;
    }
    __syncthreads();
    lv = slv;
    pdl_wait();
  }
  auto barrier = [&]() {
    if constexpr (ONE) {
      __syncthreads();
    } else {
      grid_barrier(gb);
    }
  };
  // ---- down
  for (int l = 0; l + 1 < nlev; ++l) {
    const TailLevel<T>& F = lv[l];
    const TailLevel<T>& C = lv[l + 1];
    const LevelView<T> FL = F.L;
    T* __restrict__ Fx = F.x;
    const T* __restrict__ Fb = F.b;
    for (int g = tid; g < FL.N; g += nth) Fx[g] = FL.dinv[g] * Fb[g];
    for (int base = 0; base < FL.nr; base += nth / FL.tpr)
      u_row_sum<false>(
          FL, base + tid / FL.tpr, tid % FL.tpr, [&](int col, int) { return FL.dinv[col]; },
          [&](int col, int, T d) { return d * Fb[col]; });
    barrier();
    T* __restrict__ Fr = F.r;
    for (int g = tid; g < FL.N; g += nth) {
      const DPart& sp = FL.parts[tail_part(FL.cellstart, FL.np, g)];
      Fr[g] = Fb[g] - tail_apply(FL, sp, Fx, g - sp.off, F.shape);
    }
    barrier();
    const LevelView<T> CL = C.L;
    T* __restrict__ Cb = C.b;
    for (int gc = tid; gc < CL.N; gc += nth) {
      const int p = tail_part(CL.cellstart, CL.np, gc);
      const DPart& fp = FL.parts[p];
      const DPart& cp = CL.parts[p];
      int cc = gc - cp.off;
      int I[3];
      cell_coords(cp, cc, I[0], I[1], I[2]);
      const int d = fp.dstar;
      T v;
      if (d < 0) {
        v = Fr[fp.off + (I[2] * fp.n[1] + I[1]) * fp.n[0] + I[0]];
      } else {
        int f[3] = {I[0], I[1], I[2]};
        const int anchor = 2 * I[d] + fp.par;
        f[d] = anchor;
        const int sd = (d == 0) ? 1 : (d == 1 ? fp.n[0] : fp.n[0] * fp.n[1]);
        const int fa = fp.off + (f[2] * fp.n[1] + f[1]) * fp.n[0] + f[0];
        v = Fr[fa];
        if (anchor - 1 >= 0) {
          f[d] = anchor - 1;
          v = fma(FL.Pe[fp.poff + fine_point_index(fp, f[0], f[1], f[2])], Fr[fa - sd], v);
        }
        if (anchor + 1 < fp.n[d]) {
          f[d] = anchor + 1;
          v = fma(FL.Pw[fp.poff + fine_point_index(fp, f[0], f[1], f[2])], Fr[fa + sd], v);
        }
      }
      Cb[gc] = v;
    }
    barrier();
  }
  // ---- coarsest level
  {
    const TailLevel<T>& Lc = lv[nlev - 1];
    if (coarse_direct) {
      for (int i = tid; i < nL; i += nth) {
        const double* row = cinv + (long long)i * nL;
        double s0 = 0.0, s1 = 0.0;
        int jj = 0;
        for (; jj + 1 < nL; jj += 2) {
          s0 = fma(row[jj], (double)Lc.b[jj], s0);
          s1 = fma(row[jj + 1], (double)Lc.b[jj + 1], s1);
        }
        if (jj < nL) s0 = fma(row[jj], (double)Lc.b[jj], s0);
        Lc.x[i] = (T)(s0 + s1);
      }
    } else {
      for (int g = tid; g < Lc.L.N; g += nth) Lc.x[g] = Lc.L.dinv[g] * Lc.b[g];
    }
    barrier();
  }
  // ---- up
  const T* e = lv[nlev - 1].x;
  for (int l = nlev - 2; l >= 0; --l) {
    const TailLevel<T>& F = lv[l];
    const LevelView<T> FL = F.L;
    const T* __restrict__ Fx = F.x;
    T* __restrict__ Fr = F.r;
    for (int g = tid; g < FL.N; g += nth) {
      const DPart& fp = FL.parts[tail_part(FL.cellstart, FL.np, g)];
      int c = g - fp.off, i, j, k;
      cell_coords(fp, c, i, j, k);
      Fr[g] = add_p_row(Fx[g], p_row(fp, FL.Pw, FL.Pe, i, j, k), e);
    }
    for (int base = 0; base < FL.nr; base += nth / FL.tpr)
      u_row_sum<false>(
          FL, base + tid / FL.tpr, tid % FL.tpr,
          [&](int, int q) {
            return PCol<T>{FL.u_pj[2 * q], FL.u_pj[2 * q + 1], FL.u_pw[2 * q], FL.u_pw[2 * q + 1]};
          },
          [&](int col, int, const PCol<T>& pc) {
            T v = Fx[col];
            if (pc.j0 >= 0) v = fma(pc.w0, e[pc.j0], v);
            if (pc.j1 >= 0) v = fma(pc.w1, e[pc.j1], v);
            return v;
          });
    barrier();
    T* __restrict__ Ft = F.t;
    const T* __restrict__ Fb = F.b;
    for (int g = tid; g < FL.N; g += nth) {
      const DPart& sp = FL.parts[tail_part(FL.cellstart, FL.np, g)];
      Ft[g] = fma(FL.dinv[g], Fb[g] - tail_apply(FL, sp, Fr, g - sp.off, F.shape), Fr[g]);
    }
    barrier();
    e = Ft;
  }
}

// Coarsest level with the explicit inverse: x = A_L^-1 b, one thread per row.
template <class T>
__global__ void k_coarse_apply(int n, const double* inv, const T* b,
                               T* x) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ double sb[];
  for (int i = threadIdx.x; i < n; i += blockDim.x) sb[i] = (double)b[i];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double* row = inv + (long long)i * n;
    double s0 = 0.0, s1 = 0.0;
    int jj = 0;
    for (; jj + 1 < n; jj += 2) {
      s0 = fma(row[jj], sb[jj], s0);
      s1 = fma(row[jj + 1], sb[jj + 1], s1);
    }
    if (jj < n) s0 = fma(row[jj], sb[jj], s0);
    x[i] = (T)(s0 + s1);
  }
}

// inv = (L L^T)^-1, one thread per column.
__global__ void k_coarse_inverse(int n, const double* __restrict__ Lf, double* __restrict__ inv) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    // forward: L y = e_j, stored in column j of inv
    for (int i = 0; i < n; ++i) {
      double s0 = (i == j) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s0 -= Lf[(long long)i * n + k] * inv[(long long)k * n + j];
      inv[(long long)i * n + j] = s0 / Lf[(long long)i * n + i];
    }
    // backward: L^T z = y
    for (int i = n - 1; i >= 0; --i) {
      double s0 = inv[(long long)i * n + j];
      for (int k = i + 1; k < n; ++k) s0 -= Lf[(long long)k * n + i] * inv[(long long)k * n + j];
      inv[(long long)i * n + j] = s0 / Lf[(long long)i * n + i];
    }
  }
}

__global__ void k_cast_d2f(const double* in, float* out, int n) {
  pdl_trigger();
  pdl_wait();
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) out[g] = (float)in[g];
}
__global__ void k_fill(double* x, long long n, double v) {
  pdl_trigger();
  pdl_wait();
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n;
       g += (long long)gridDim.x * blockDim.x)
    x[g] = v;
}

__global__ void k_cast_f2d(const float* in, double* out, int n) {
  pdl_trigger();
  pdl_wait();
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) out[g] = (double)in[g];
}

__global__ void __launch_bounds__(NT, 4) k_matvec(LevelView<double> L, const double* x,
                                               double* y, int padded) {
  pdl_trigger();
  __shared__ DPart sp;
  int p = block_part(L.blk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  TILE_LOOP(c, sp) {
    int i, j, k;
    cell_coords(sp, c, i, j, k);
    y[sp.off + c] = apply_A_sh<SH_CHECKED>(L, sp, x, c);
  }
}

// ---------------------------------------------------------------------------
// PCG (FP64), one instance per problem of the solver: a single problem, or a
// batch of independent problems that share one hierarchy.  Every vector
// kernel runs over the level-0 cell tiles, so each block belongs to one part
// and hence one problem (DPart::prob); the level-0 blocks of problem k are
// pb[k] .. pb[k+1]-1.  A dot product is a partial sum per block plus one
// final sum per problem in a fixed order (bitwise reproducible).  Once a
// problem has stopped (sc[k].done) its x and r no longer change.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void finish_sums(const double* __restrict__ partial, int b0, int b1,
                                            double* out) {
  __shared__ double sh[NT];
  for (int q = 0; q < K; ++q) {
    double s = 0.0;
    for (int b = b0 + threadIdx.x; b < b1; b += NT) s += partial[(long long)K * b + q];
    double r = block_sum<NT>(s, sh);
    if (threadIdx.x == 0) out[q] = r;
  }
}

// r = b - A x; partial sums of (b.b, r.r)
template <int SH>
__global__ void __launch_bounds__(NT, 4) k_pcg_init(LevelView<double> L, const double* b,
                                                 const double* x, double* r,
                                                 double* partial) {
  pdl_trigger();
  __shared__ DPart sp;
  __shared__ double sh[NT];
  block_part(L.blk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  double bb = 0.0, rr = 0.0;
  TILE_LOOP(c, sp) {
    int g = sp.off + c;
    double bv = b[g];
    double rv = bv - apply_A_sh<SH>(L, sp, x, c);
    r[g] = rv;
    bb = fma(bv, bv, bb);
    rr = fma(rv, rv, rr);
  }
  double s0 = block_sum<NT>(bb, sh);
  double s1 = block_sum<NT>(rr, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s0;
    partial[2 * blockIdx.x + 1] = s1;
  }
}

// per problem (one block each): ||b||^2, ||r||^2 and the stopping threshold
__global__ void __launch_bounds__(NT) k_pcg_init_fin(const double* partial,
                                                     const int* pb, PcgScalars* sc,
                                                     double* hist, int hstride) {
  pdl_trigger();
  pdl_wait();
  __shared__ double out[2];
  const int k = blockIdx.x;
  finish_sums<2>(partial, pb[k], pb[k + 1], out);
  if (threadIdx.x == 0) {
    PcgScalars& S = sc[k];
    S.bb = out[0];
    S.rr = out[1];
    S.tol2bb = S.tol * S.tol * out[0];
    S.iter = 0;
    if (hist) hist[(long long)k * hstride] = out[1];
    S.status = 0;
    S.done = (out[1] <= S.tol2bb) ? 1 : 0;
  }
}

// p = z (and zprev = z for flexible CG); partial r.z
__global__ void __launch_bounds__(NT) k_pcg_start(LevelView<double> L, const double* r,
                                                  const double* z,
                                                  double* p, double* zprev,
                                                  int flex, double* partial) {
  pdl_trigger();
  __shared__ DPart sp;
  __shared__ double sh[NT];
  block_part(L.blk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  double s = 0.0;
  TILE_LOOP(c, sp) {
    const int g = sp.off + c;
    const double zv = z[g];
    p[g] = zv;
    if (flex) zprev[g] = zv;
    s = fma(r[g], zv, s);
  }
  double t = block_sum<NT>(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__device__ __forceinline__ void set_continue(int active, cudaGraphConditionalHandle h,
                                             int use_handle) {
  if (use_handle) cudaGraphSetConditional(h, active ? 1u : 0u);
}

__global__ void __launch_bounds__(NT) k_pcg_start_fin(const double* partial,
                                                      const int* pb, PcgScalars* sc) {
  pdl_trigger();
  pdl_wait();
  __shared__ double out[1];
  const int k = blockIdx.x;
  finish_sums<1>(partial, pb[k], pb[k + 1], out);
  PcgScalars& S = sc[k];
  if (threadIdx.x == 0 && !S.done) {
    S.rz = out[0];
    if (!(out[0] > 0.0) || !isfinite(out[0])) {
      S.status = SSAMG_ERR_BREAKDOWN;
      S.done = 1;
    }
  }
}

// partial (r.z, r.zprev) for beta; zprev takes the new z (flexible CG)
__global__ void __launch_bounds__(NT) k_pcg_dots_rz(LevelView<double> L,
                                                    const double* r,
                                                    const double* z,
                                                    double* zprev, int flex,
                                                    double* partial) {
  pdl_trigger();
  __shared__ DPart sp;
  __shared__ double sh[NT];
  block_part(L.blk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  double s0 = 0.0, s1 = 0.0;
  TILE_LOOP(c, sp) {
    const int g = sp.off + c;
    const double rv = r[g], zv = z[g];
    s0 = fma(rv, zv, s0);
    if (flex) {
      s1 = fma(rv, zprev[g], s1);
      zprev[g] = zv;
    }
  }
  double t0 = block_sum<NT>(s0, sh);
  double t1 = block_sum<NT>(s1, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = t0;
    partial[2 * blockIdx.x + 1] = t1;
  }
}

__global__ void __launch_bounds__(NT) k_pcg_beta_fin(const double* partial,
                                                     const int* pb, PcgScalars* sc) {
  pdl_trigger();
  pdl_wait();
  __shared__ double out[2];
  const int k = blockIdx.x;
  finish_sums<2>(partial, pb[k], pb[k + 1], out);
  PcgScalars& S = sc[k];
  if (threadIdx.x == 0 && !S.done) {
    double rz = out[0];
    double num = S.flexible ? (rz - out[1]) : rz;
    S.beta = num / S.rz;
    S.rz = rz;
    if (!isfinite(rz) || !isfinite(S.beta)) {
      S.status = SSAMG_ERR_BREAKDOWN;
      S.done = 1;
    }
  }
}

// p = z + beta p (per problem)
__global__ void __launch_bounds__(NT) k_pcg_xpby(LevelView<double> L, const double* z,
                                                 double* p,
                                                 const PcgScalars* sc) {
  pdl_trigger();
  __shared__ DPart sp;
  block_part(L.blk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  const PcgScalars& S = sc[sp.prob];
  if (S.done) return;
  const double beta = S.beta;
  TILE_LOOP(c, sp) {
    const int g = sp.off + c;
    p[g] = fma(beta, p[g], z[g]);
  }
}

// q = A p; partial p.q
template <int SH>
__global__ void __launch_bounds__(NT, 4) k_pcg_spmv_dot(LevelView<double> L, const double* p,
                                                     double* q,
                                                     double* partial) {
  pdl_trigger();
  __shared__ DPart sp;
  __shared__ double sh[NT];
  block_part(L.blk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  double s = 0.0;
  TILE_LOOP(c, sp) {
    int g = sp.off + c;
    double qv = apply_A_sh<SH>(L, sp, p, c);
    q[g] = qv;
    s = fma(p[g], qv, s);
  }
  double t = block_sum<NT>(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(NT) k_pcg_alpha_fin(const double* partial,
                                                      const int* pb, PcgScalars* sc) {
  pdl_trigger();
  pdl_wait();
  __shared__ double out[1];
  const int k = blockIdx.x;
  finish_sums<1>(partial, pb[k], pb[k + 1], out);
  PcgScalars& S = sc[k];
  if (threadIdx.x == 0 && !S.done) {
    double pq = out[0];
    S.pq = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
      S.status = SSAMG_ERR_BREAKDOWN;
      S.done = 1;
      S.alpha = 0.0;
    } else {
      S.alpha = S.rz / pq;
    }
  }
}

// x += alpha p; r -= alpha q; partial r.r (per problem)
__global__ void __launch_bounds__(NT) k_pcg_update(LevelView<double> L, const double* p,
                                                   const double* q,
                                                   double* x, double* r,
                                                   double* partial,
                                                   const PcgScalars* sc) {
  pdl_trigger();
  __shared__ DPart sp;
  __shared__ double sh[NT];
  block_part(L.blk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  const PcgScalars& S = sc[sp.prob];
  if (S.done) return;  // the problem's final sum ignores this block's partial
  const double alpha = S.alpha;
  double s = 0.0;
  TILE_LOOP(c, sp) {
    const int g = sp.off + c;
    x[g] = fma(alpha, p[g], x[g]);
    const double rv = fma(-alpha, q[g], r[g]);
    r[g] = rv;
    s = fma(rv, rv, s);
  }
  double t = block_sum<NT>(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// Per problem: ||r||^2, iteration count and the stopping test.  The last
// block to finish (ticket counter) sets ctl->active to whether any problem
// still iterates and, inside the solve graph, the loop condition with it.
__global__ void __launch_bounds__(NT) k_pcg_update_fin(const double* partial,
                                                       const int* pb, PcgScalars* sc,
                                                       PcgCtl* ctl, cudaGraphConditionalHandle h,
                                                       int use_handle, double* hist,
                                                       int hstride, const PcgScalars* any_sc,
                                                       int any_n) {
  pdl_trigger();
  pdl_wait();
  __shared__ double out[1];
  __shared__ bool last;
  const int k = blockIdx.x;
  PcgScalars& S = sc[k];
  const bool was_done = S.done;
  finish_sums<1>(partial, pb[k], pb[k + 1], out);
  if (threadIdx.x == 0) {
    if (!was_done) {
      S.rr = out[0];
      S.iter += 1;
      if (hist && S.iter < hstride) hist[(long long)k * hstride + S.iter] = out[0];
      if (!isfinite(out[0])) S.status = SSAMG_ERR_BREAKDOWN;
      if (S.status != 0 || out[0] <= S.tol2bb || S.iter >= S.max_iter) S.done = 1;
    }
    __threadfence();
    last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    // any problem of any right-hand side solved together (the last
    // right-hand side's launch sees them all updated and decides)
    int active = 0;
    for (int q = 0; q < any_n; ++q)
      active |= !*reinterpret_cast<volatile const int*>(&any_sc[q].done);
    ctl->ticket = 0;
    ctl->active = active;
    set_continue(active, h, use_handle);
  }
}

// per problem: (||b||^2, ||b - A x||^2)
__global__ void __launch_bounds__(NT) k_true_res_fin(const double* partial,
                                                     const int* pb,
                                                     double* out) {
  pdl_trigger();
  pdl_wait();
  __shared__ double o2[2];
  const int k = blockIdx.x;
  finish_sums<2>(partial, pb[k], pb[k + 1], o2);
  if (threadIdx.x == 0) {
    out[2 * k] = o2[0];
    out[2 * k + 1] = o2[1];
  }
}

// ---------------------------------------------------------------------------
// Differentiation
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_coef_gradient(LevelView<double> L,
                                                      const double* lam,
                                                      const double* x,
                                                      double* dcoef, long long N) {
  pdl_trigger();
  __shared__ DPart sp;
  int p = block_part(L.blk, L.parts, L.np, sp);
  __syncthreads();
  pdl_wait();
  TILE_LOOP(c, sp) {
    int i, j, k;
    cell_coords(sp, c, i, j, k);
    int g = sp.off + c;
    double l = lam[g];
    for (int e = 0; e < sp.nent; ++e) {
      double v = 0.0;
      if (inside(sp, i + sp.o[e][0], j + sp.o[e][1], k + sp.o[e][2])) v = -l * x[g + sp.disp[e]];
      dcoef[(long long)sp.uent[e] * N + g] = v;  // in the user's entry order
    }
  }
}

// kappa = exp(g), once per cell (FP64 exp is the expensive step on this GPU;
// the gradient reads each cell's kappa up to seven times).
__global__ void __launch_bounds__(NT) k_exp(int n, const double* gg, double* kap) {
  pdl_trigger();
  pdl_wait();
  const int c = blockIdx.x * NT + threadIdx.x;
  if (c < n) kap[c] = exp(gg[c]);
}

__global__ void __launch_bounds__(NT) k_diffusion_exp_gradient(LevelView<double> L,
                                                               const double* kap,
                                                               const double* lam,
                                                               const double* x,
                                                               double* dg) {
  pdl_trigger();
  pdl_wait();
  __shared__ DPart sp;
  stage_part(sp, L.parts);
  __syncthreads();
  int c = blockIdx.x * NT + threadIdx.x;
  if (c >= sp.ncell) return;
  int i, j, k;
  cell_coords(sp, c, i, j, k);
  const double kc = kap[c];
  const double lc = lam[c], xc = x[c];
  const int sx = 1, sy = sp.n[0], sz = sp.n[0] * sp.n[1];
  double acc = 0.0;
  // faces -x, +x, -y, +y, -z, +z
  auto face = [&](bool in, int d) {
    if (in) {
      const double kn = kap[c + d];
      const double s = kc + kn;
      const double dt = 2.0 * kn * kn / (s * s);
      acc -= dt * (lc - lam[c + d]) * (xc - x[c + d]);
    } else {
      acc -= lc * xc;
    }
  };
  face(i > 0, -sx);
  face(i < sp.n[0] - 1, sx);
  face(j > 0, -sy);
  face(j < sp.n[1] - 1, sy);
  face(k > 0, -sz);
  face(k < sp.n[2] - 1, sz);
  dg[c] = kc * acc;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
namespace {
// Launch of a solve kernel: with programmatic stream serialisation when the
// calling entry point enables it (see pdl_wait), else a plain launch.
template <typename... P, typename... A>
void launch_k(void (*kern)(P...), int grid, int block, size_t smem, cudaStream_t st, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = g_ssamg_pdl ? 1 : 0;
  SSAMG_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...));
}
}  // namespace

// Restriction onto / prolongation on L over bricks: levels with at least
// SSAMG_RP_BRICKS bricks (at least a block per SM) that the parts fill
// to SSAMG_RP_FILL (small or uneven parts leave bricks partly idle), unless
// the tile table keeps the level on cell tiles.
bool rp_bricks(const Level& L) {
  return g_ssamg_bricks && L.bricks && L.nbblk >= SSAMG_RP_BRICKS &&
         L.brick_fill >= SSAMG_RP_FILL;
}

bool uses_bricks(const Level& L) {
  return g_ssamg_bricks && L.bricks && L.shape == SH_K7 && L.nbblk > 0;
}

// Level-0 block ranges of the problems for the partials that L's operator
// apply launches write (brick or cell-tile blocks).
const int* partial_ranges(const Level& L, const PcgCtx& c) { return uses_bricks(L) ? c.pbb : c.pb; }
const int* final_ranges(const Level& L, const PcgCtx& c) { return uses_bricks(L) ? c.pbb : c.pb; }

template <class T>
void launch_relax0(const Level& L, const T* b, T* x, cudaStream_t st) {
  const T* dinv = L.view<T>().dinv;
  launch_k(k_relax0<T>, cdiv(L.N, NT), NT, 0, st, (int)L.N, dinv, b, x);
  SSAMG_LAUNCH_CHECK();
}
template <class T>
void launch_relax0_u(const Level& L, const T* b, T* x, cudaStream_t st) {
  int nb = cdiv(L.N, NT * SSAMG_EW);
  launch_k(k_relax0_u<T>, nb + L.nublk, NT, 0, st, L.view<T>(), nb, b, x);
  SSAMG_LAUNCH_CHECK();
}
// one group of g right-hand sides (g = 1 .. SSAMG_RHS_GROUP) of shape SHC
#define RHS_GROUP_LAUNCH(SHC)                                                               \
  switch (g) {                                                                             \
    case 1: launch_k(k_cycle_r<T, SHC, 1, RELAX>, L.nblk, NT, 0, st, v, xg, bg, og); break; \
    case 2: launch_k(k_cycle_r<T, SHC, 2, RELAX>, L.nblk, NT, 0, st, v, xg, bg, og); break; \
    case 3: launch_k(k_cycle_r<T, SHC, 3, RELAX>, L.nblk, NT, 0, st, v, xg, bg, og); break; \
    default: launch_k(k_cycle_r<T, SHC, 4, RELAX>, L.nblk, NT, 0, st, v, xg, bg, og); break; \
  }
#define SH_DISPATCH(shape, KCALL)                         \
  switch (shape) {                                        \
    case SH_U7: { constexpr int SHV = SH_U7; KCALL; } break;   \
    case SH_U15: { constexpr int SHV = SH_U15; KCALL; } break; \
    case SH_C27: { constexpr int SHV = SH_C27; KCALL; } break; \
    case SH_UGEN: { constexpr int SHV = SH_UGEN; KCALL; } break; \
    case SH_K7: { constexpr int SHV = SH_K7; KCALL; } break;   \
    default: { constexpr int SHV = SH_CHECKED; KCALL; } break; \
  }

template <class T>
void launch_relax0_u_first(const Level& L, const double* r64, T* b0, T* x, cudaStream_t st) {
  int nb = cdiv(L.N, NT * SSAMG_EW);
  launch_k(k_relax0_u_first<T>, nb + L.nublk, NT, 0, st, L.view<T>(), nb, r64, b0, x);
  SSAMG_LAUNCH_CHECK();
}
template <class T>
void launch_relax_final(const Level& L, const T* x, const T* b, double* z, const double* rpcg,
                        double* zprev, double* partial, cudaStream_t st) {
  // zprev may be null (no flexible CG): pass a valid buffer and a flag
  const int flex = zprev != nullptr;
  double* zp = flex ? zprev : z;
  if (uses_bricks(L))
    launch_k(pick_km(L.kvar, k7b_relax_final<T, 0>, k7b_relax_final<T, 1>, k7b_relax_final<T, 2>),
             L.nbblk, NT, 0, st, L.view<T>(), x, b, z, rpcg, zp, flex, partial);
  else
    SH_DISPATCH(L.shape, (launch_k(k_relax_final<T, SHV>, L.nblk, NT, 0, st, L.view<T>(), x, b, z,
                                   rpcg, zp, flex, partial)));
  SSAMG_LAUNCH_CHECK();
}
template <class T>
void launch_prolong_u(const Level& F, const T* ec, const T* xin, T* xout, cudaStream_t st) {
  if (rp_bricks(F)) {
    launch_k(k_prolong_ub<T>, 2 * F.nbblk + F.nublk, NT, 0, st, F.view<T>(), ec, xin, xout,
             2 * F.nbblk);
  } else {
    launch_k(k_prolong_u<T>, F.nblk + F.nublk, NT, 0, st, F.view<T>(), ec, xin, xout, F.nblk);
  }
  SSAMG_LAUNCH_CHECK();
}
template <class T>
void launch_uy(const Level& L, const T* x, cudaStream_t st) {
  if (L.nublk == 0) return;
  launch_k(k_uy<T>, L.nublk, NT, 0, st, L.view<T>(), x);
  SSAMG_LAUNCH_CHECK();
}

template <class T>
void launch_residual(const Level& L, const T* x, const T* b, T* r, cudaStream_t st) {
  if (uses_bricks(L))
    launch_k(pick_km(L.kvar, k7b_residual<T, 0>, k7b_residual<T, 1>, k7b_residual<T, 2>), L.nbblk, NT, 0,
             st, L.view<T>(), x, b, r);
  else
    SH_DISPATCH(L.shape, (launch_k(k_residual<T, SHV>, L.nblk, NT, 0, st, L.view<T>(), x, b, r)));
  SSAMG_LAUNCH_CHECK();
}
template <class T>
void launch_relax(const Level& L, const T* x, const T* b, T* xo, cudaStream_t st) {
  if (uses_bricks(L))
    launch_k(pick_km(L.kvar, k7b_relax<T, 0>, k7b_relax<T, 1>, k7b_relax<T, 2>), L.nbblk, NT, 0,
             st, L.view<T>(), x, b, xo);
  else
    SH_DISPATCH(L.shape, (launch_k(k_relax<T, SHV>, L.nblk, NT, 0, st, L.view<T>(), x, b, xo)));
  SSAMG_LAUNCH_CHECK();
}
// R right-hand sides (cell-tile levels only): vectors and U x of right-hand
// side j at + j vstride, its scalars at skip + j skip_stride.  Shapes with
// every entry per cell take up to SSAMG_RHS_GROUP right-hand sides per thread
// (one launch per group); the others one launch with R blocks per tile, side
// by side, so that a tile's coefficients come from HBM once.
template <class T, bool RELAX>
void launch_cycle_rhs(const Level& L, int R, long long vstride, int skip_stride, const T* x,
                      const T* b, T* out, cudaStream_t st) {
  if (shape_has_rhs_form(L.shape)) {
    for (int j0 = 0; j0 < R; j0 += SSAMG_RHS_GROUP) {
      const int g = std::min(SSAMG_RHS_GROUP, R - j0);
      LevelView<T> v = L.view<T>();
      v.vstride = vstride;
      v.skip_stride = skip_stride;
      const long long o = (long long)j0 * vstride;
      if (v.uy) v.uy += o;
      if (v.skip) v.skip += (long long)j0 * skip_stride;
      const T* xg = x + o;
      const T* bg = b + o;
      T* og = out + o;
      switch (L.shape) {
        case SH_U7: RHS_GROUP_LAUNCH(SH_U7); break;
        case SH_U15: RHS_GROUP_LAUNCH(SH_U15); break;
        case SH_C27: RHS_GROUP_LAUNCH(SH_C27); break;
        default: RHS_GROUP_LAUNCH(SH_UGEN); break;
      }
      SSAMG_LAUNCH_CHECK();
    }
    return;
  }
  LevelView<T> v = L.view<T>();
  v.nrhs = R;
  v.vstride = vstride;
  v.skip_stride = skip_stride;
  if constexpr (RELAX) {
    SH_DISPATCH(L.shape, (launch_k(k_relax<T, SHV>, L.nblk * R, NT, 0, st, v, x, b, out)));
  } else {
    SH_DISPATCH(L.shape, (launch_k(k_residual<T, SHV>, L.nblk * R, NT, 0, st, v, x, b, out)));
  }
  SSAMG_LAUNCH_CHECK();
}
template <class T>
void launch_residual_rhs(const Level& L, int R, long long vstride, int skip_stride, const T* x,
                         const T* b, T* r, cudaStream_t st) {
  launch_cycle_rhs<T, false>(L, R, vstride, skip_stride, x, b, r, st);
}
template <class T>
void launch_relax_rhs(const Level& L, int R, long long vstride, int skip_stride, const T* x,
                      const T* b, T* xo, cudaStream_t st) {
  launch_cycle_rhs<T, true>(L, R, vstride, skip_stride, x, b, xo, st);
}
template <class T>
void launch_restrict(const Level& F, const Level& Cl, const T* r, T* bc, T* xc, cudaStream_t st) {
  // with xc: also x = omega M^-1 b on the coarse level, and its U x row jobs
  const int nrow = xc ? Cl.nublk : 0;
  if (rp_bricks(Cl)) {
    launch_k(k_restrict_b<T>, Cl.nbblk + nrow, NT, 0, st, F.view<T>(), Cl.view<T>(), r, bc, xc,
             Cl.nbblk);
  } else {
    launch_k(k_restrict<T>, Cl.nblk + nrow, NT, 0, st, F.view<T>(), Cl.view<T>(), r, bc, xc,
             Cl.nblk);
  }
  SSAMG_LAUNCH_CHECK();
}
template <class T>
void launch_prolong(const Level& F, const Level& Cl, const T* ec, T* x, cudaStream_t st) {
  (void)Cl;
  launch_k(k_prolong<T>, F.nblk, NT, 0, st, F.view<T>(), ec, x);
  SSAMG_LAUNCH_CHECK();
}
template <class T>
void launch_coarse_solve(int n, const double* Lfac, const T* b, T* x, cudaStream_t st) {
  const int staged = (n + n * n) * (int)sizeof(double) <= 40 * 1024;
  size_t sm = sizeof(double) * (staged ? n + n * n : n);
  launch_k(k_coarse_solve<T>, 1, 32, sm, st, n, Lfac, b, x, staged);
  SSAMG_LAUNCH_CHECK();
}

template <class T>
void launch_coarse_apply(int n, const double* inv, const T* b, T* x, cudaStream_t st) {
  launch_k(k_coarse_apply<T>, 1, 256, sizeof(double) * n, st, n, inv, b, x);
  SSAMG_LAUNCH_CHECK();
}

template <class T>
size_t vtail_one_smem(int nlev, int nparts) {
  return sizeof(TailLevel<T>) * nlev + sizeof(DPart) * nparts;
}

template <class T>
bool vtail_one_prepare(int nlev, int nparts) {
  const size_t sm = vtail_one_smem<T>(nlev, nparts);
  if (sm > 200 * 1024) return false;
  SSAMG_CUDA(cudaFuncSetAttribute(k_vtail<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm));
  return true;
}

template <class T>
void launch_vtail(const TailLevel<T>* lv, int nlev, const double* cinv, int nL, int coarse_direct,
                  int nblocks, TailBarrier* gb, cudaStream_t st, int nparts) {
  if (nblocks == 0) {  // single CTA
    launch_k(k_vtail<T, true>, 1, SSAMG_TAIL_CTA, vtail_one_smem<T>(nlev, nparts), st, lv, nlev,
             cinv, nL, coarse_direct, gb);
    SSAMG_LAUNCH_CHECK();
    return;
  }
  SSAMG_CUDA(cudaMemsetAsync(gb, 0, sizeof(unsigned), st));  // counter (err is sticky)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(TB);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SSAMG_CUDA(cudaLaunchKernelEx(&cfg, k_vtail<T, false>, lv, nlev, cinv, nL, coarse_direct, gb));
  SSAMG_LAUNCH_CHECK();
}

int barrier_selftest(int nblocks, int extra, unsigned cap, cudaStream_t st) {
  TailBarrier* gb = nullptr;
  SSAMG_CUDA(cudaMalloc(&gb, sizeof(TailBarrier)));
  const TailBarrier init{0u, cap, 0, extra};
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(gb, &init, sizeof(init), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(32);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_barrier_selftest, gb);
    if (e == cudaSuccess) ++g_ssamg_launches;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &gb->err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(gb);
  SSAMG_CUDA(e);
  return err;
}

int tail_max_blocks() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_vtail<float, false>, TB, 0);
  int per2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_vtail<double, false>, TB, 0);
  return sms * std::min(per, per2);
}

void launch_coarse_inverse(int n, const double* Lfac, double* inv, cudaStream_t st) {
  k_coarse_inverse<<<cdiv(n, 64), 64, 0, st>>>(n, Lfac, inv);
  SSAMG_LAUNCH_CHECK();
}

#define INST(T)                                                                            \
  template void launch_relax0<T>(const Level&, const T*, T*, cudaStream_t);                \
  template void launch_relax0_u<T>(const Level&, const T*, T*, cudaStream_t);              \
  template void launch_prolong_u<T>(const Level&, const T*, const T*, T*, cudaStream_t);   \
  template void launch_relax0_u_first<T>(const Level&, const double*, T*, T*, cudaStream_t); \
  template void launch_relax_final<T>(const Level&, const T*, const T*, double*, const double*, \
                                      double*, double*, cudaStream_t);                     \
  template void launch_uy<T>(const Level&, const T*, cudaStream_t);                        \
  template void launch_vtail<T>(const TailLevel<T>*, int, const double*, int, int, int,      \
                                TailBarrier*, cudaStream_t, int);                          \
  template bool vtail_one_prepare<T>(int, int);                                            \
  template void launch_coarse_apply<T>(int, const double*, const T*, T*, cudaStream_t);    \
  template void launch_residual<T>(const Level&, const T*, const T*, T*, cudaStream_t);    \
  template void launch_relax<T>(const Level&, const T*, const T*, T*, cudaStream_t);       \
  template void launch_residual_rhs<T>(const Level&, int, long long, int, const T*, const T*, \
                                       T*, cudaStream_t);                                    \
  template void launch_relax_rhs<T>(const Level&, int, long long, int, const T*, const T*,    \
                                    T*, cudaStream_t);                                       \
  template void launch_restrict<T>(const Level&, const Level&, const T*, T*, T*, cudaStream_t); \
  template void launch_prolong<T>(const Level&, const Level&, const T*, T*, cudaStream_t);  \
  template void launch_coarse_solve<T>(int, const double*, const T*, T*, cudaStream_t);
INST(float)
INST(double)
#undef INST

void launch_cast_d2f(const double* in, float* out, long long n, cudaStream_t st) {
  launch_k(k_cast_d2f, cdiv(n, NT), NT, 0, st, in, out, (int)n);
  SSAMG_LAUNCH_CHECK();
}
void launch_fill(double* x, long long n, double v, cudaStream_t st) {
  launch_k(k_fill, (int)std::min<long long>(cdiv(n, NT), 8 * 152), NT, 0, st, x, n, v);
  SSAMG_LAUNCH_CHECK();
}
void launch_cast_f2d(const float* in, double* out, long long n, cudaStream_t st) {
  launch_k(k_cast_f2d, cdiv(n, NT), NT, 0, st, in, out, (int)n);
  SSAMG_LAUNCH_CHECK();
}
void launch_matvec(const Level& L, const double* x, double* y, cudaStream_t st) {
  launch_uy<double>(L, x, st);
  launch_k(k_matvec, L.nblk, NT, 0, st, L.view<double>(), x, y, 0);
  SSAMG_LAUNCH_CHECK();
}

void launch_pcg_init(const Level& L, const double* b, const double* x, double* r,
                     const PcgCtx& c, cudaStream_t st) {
  launch_uy<double>(L, x, st);
  if (uses_bricks(L))
    launch_k(pick_km(L.kvar, k7b_pcg_init<0>, k7b_pcg_init<1>, k7b_pcg_init<2>), L.nbblk, NT, 0,
             st, L.view<double>(), b, x, r, c.partial);
  else
    SH_DISPATCH(L.shape, (launch_k(k_pcg_init<SHV>, L.nblk, NT, 0, st, L.view<double>(), b, x, r,
                                   c.partial)));
  SSAMG_LAUNCH_CHECK();
  launch_k(k_pcg_init_fin, c.nprob, NT, 0, st, c.partial, partial_ranges(L, c), c.sc, c.hist,
           c.hstride);
  SSAMG_LAUNCH_CHECK();
}

void launch_pcg_start(const Level& L0, const double* r, const double* z, double* p, double* zprev,
                      const PcgCtx& c, cudaStream_t st) {
  // zprev may be null (no flexible CG): pass a valid buffer and a flag
  launch_k(k_pcg_start, L0.nblk, NT, 0, st, L0.view<double>(), r, z, p, zprev ? zprev : p,
           zprev != nullptr, c.partial);
  SSAMG_LAUNCH_CHECK();
  launch_k(k_pcg_start_fin, c.nprob, NT, 0, st, c.partial, c.pb, c.sc);
  SSAMG_LAUNCH_CHECK();
}

void launch_pcg_beta(const Level& L0, const double* r, const double* z, double* zprev, double* p,
                     const PcgCtx& c, cudaStream_t st) {
  launch_k(k_pcg_dots_rz, L0.nblk, NT, 0, st, L0.view<double>(), r, z, zprev ? zprev : p,
           zprev != nullptr, c.partial);
  SSAMG_LAUNCH_CHECK();
  launch_pcg_beta_from_partials(L0, z, p, c, c.pb, st);
}

void launch_pcg_beta_from_partials(const Level& L0, const double* z, double* p, const PcgCtx& c,
                                   const int* ranges, cudaStream_t st) {
  launch_k(k_pcg_beta_fin, c.nprob, NT, 0, st, c.partial, ranges, c.sc);
  SSAMG_LAUNCH_CHECK();
  launch_k(k_pcg_xpby, L0.nblk, NT, 0, st, L0.view<double>(), z, p, c.sc);
  SSAMG_LAUNCH_CHECK();
}

void launch_pcg_alpha(const Level& L, const double* p, double* q, const PcgCtx& c,
                      cudaStream_t st) {
  launch_uy<double>(L, p, st);
  if (uses_bricks(L))
    launch_k(pick_km(L.kvar, k7b_spmv_dot<0>, k7b_spmv_dot<1>, k7b_spmv_dot<2>), L.nbblk, NT, 0,
             st, L.view<double>(), p, q, c.partial);
  else
    SH_DISPATCH(L.shape, (launch_k(k_pcg_spmv_dot<SHV>, L.nblk, NT, 0, st, L.view<double>(), p, q,
                                   c.partial)));
  SSAMG_LAUNCH_CHECK();
  launch_k(k_pcg_alpha_fin, c.nprob, NT, 0, st, c.partial, partial_ranges(L, c), c.sc);
  SSAMG_LAUNCH_CHECK();
}

void launch_pcg_update(const Level& L0, const double* p, const double* q, double* x, double* r,
                       const PcgCtx& c, cudaGraphConditionalHandle h, int use_handle,
                       cudaStream_t st) {
  launch_k(k_pcg_update, L0.nblk, NT, 0, st, L0.view<double>(), p, q, x, r, c.partial, c.sc);
  SSAMG_LAUNCH_CHECK();
  launch_k(k_pcg_update_fin, c.nprob, NT, 0, st, c.partial, c.pb, c.sc, c.ctl, h, use_handle,
           c.hist, c.hstride, (const PcgScalars*)c.any_sc, c.any_n);
  SSAMG_LAUNCH_CHECK();
}

void launch_true_residual(const Level& L, const double* b, const double* x, double* r,
                          const PcgCtx& c, double* out, cudaStream_t st) {
  launch_uy<double>(L, x, st);
  if (uses_bricks(L))
    launch_k(pick_km(L.kvar, k7b_pcg_init<0>, k7b_pcg_init<1>, k7b_pcg_init<2>), L.nbblk, NT, 0,
             st, L.view<double>(), b, x, r, c.partial);
  else
    SH_DISPATCH(L.shape, (launch_k(k_pcg_init<SHV>, L.nblk, NT, 0, st, L.view<double>(), b, x, r,
                                   c.partial)));
  SSAMG_LAUNCH_CHECK();
  launch_k(k_true_res_fin, c.nprob, NT, 0, st, c.partial, partial_ranges(L, c), out);
  SSAMG_LAUNCH_CHECK();
}

void launch_coef_gradient(const Level& L, const double* lam, const double* x, double* dcoef,
                          cudaStream_t st) {
  launch_k(k_coef_gradient, L.nblk, NT, 0, st, L.view<double>(), lam, x, dcoef, L.N);
  SSAMG_LAUNCH_CHECK();
}

void launch_diffusion_exp_gradient(const Level& L, const double* g, const double* lam,
                                   const double* x, double* dg, double* kap, cudaStream_t st) {
  const int n = (int)L.parts[0].ncell;
  launch_k(k_exp, cdiv(n, NT), NT, 0, st, n, g, kap);
  SSAMG_LAUNCH_CHECK();
  launch_k(k_diffusion_exp_gradient, cdiv(n, NT), NT, 0, st, L.view<double>(), (const double*)kap,
           lam, x, dg);
  SSAMG_LAUNCH_CHECK();
}
