// Device helpers shared by the kernel translation units.
#pragma once

#include "ssamg_internal.cuh"

// Cell-wise launches give each block a tile of P.cpt x SSAMG_BLOCK
// consecutive cells of one part; thread t handles cells t, t + SSAMG_BLOCK,
// ... (coalesced).  Large levels use several cells per thread to amortise
// descriptor staging and FP64 reduction trees; small levels use one, for
// more warps to hide latency.
#define TILE_LOOP(c, P) TILE_LOOP_AT(c, P, (int)blockIdx.x)
// The same for tile block B (launches of several right-hand sides).
#define TILE_LOOP_AT(c, P, B)                                                              \
  _Pragma("unroll 1") for (int c##_m = 0,                                                  \
       c = ((B) - (P).blk0) * (P).cpt * SSAMG_BLOCK + (int)threadIdx.x;                    \
       c##_m < (P).cpt && c < (P).ncell; ++c##_m, c += SSAMG_BLOCK)
// The same tiles with the SSAMG_CPT_LARGE steps unrolled and predicated, so
// that a thread issues the loads of all its cells before it consumes the
// first; for kernels light enough in registers (restriction, prolongation).
#define TILE_LOOP_UNROLLED(c, P)                                                           \
  _Pragma("unroll") for (int c##_m = 0; c##_m < SSAMG_CPT_LARGE; ++c##_m)                  \
    if (const int c = ((int)blockIdx.x - (P).blk0) * (P).cpt * SSAMG_BLOCK +               \
                      (int)threadIdx.x + c##_m * SSAMG_BLOCK;                              \
        c##_m < (P).cpt && c < (P).ncell)
#define TILE_LOOP_FINE(c, P)                                                               \
  _Pragma("unroll 1") for (int c##_m = 0,                                                  \
       c = ((int)blockIdx.x - (P).fblk0) * (P).cpt * SSAMG_BLOCK + (int)threadIdx.x;       \
       c##_m < (P).cpt && c < (P).nfine; ++c##_m, c += SSAMG_BLOCK)

// Programmatic dependent launch.  (Pointer parameters of these kernels are
// not __restrict__: a const __restrict__ kernel parameter may be read with
// invariant loads, which the compiler may move above griddepcontrol.wait,
// before the predecessor has written the data.)  The solve's kernels are launched with
// programmatic stream serialisation: a kernel may be scheduled while its
// predecessor in the stream is still running, stages what setup wrote (block
// tables, part descriptors; host copies only), and then waits in pdl_wait()
// until the predecessor has completed and its writes are visible, before it
// touches any vector of the solve.  Since every kernel waits before it
// completes, completion is transitive down the stream.  pdl_trigger() lets
// the successor be scheduled once every block of this grid has started.
// Without the launch attribute both instructions return at once.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Part owning block b of a launch whose per-part block starts are blk[0..np].
__device__ __forceinline__ int find_part(const int* __restrict__ blk, int np, int b) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(blk + mid) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Part owning global cell g of a level (cellstart[0..np]).
__device__ __forceinline__ int find_part_cell(const int* __restrict__ cs, int np, int g) {
  return find_part(cs, np, g);
}

// Part of this block (cell tiles, or fine-point tiles when `fine` -- the
// block table passed is then the fine-point one), staged in shared memory
// from the level's descriptor array.  All threads call; a barrier follows in
// the caller.
__device__ __forceinline__ int block_part(const int* __restrict__ gblk,
                                          const DPart* __restrict__ gparts, int np, DPart& sm,
                                          int tile = -1) {
  const int p = find_part(gblk, np, tile < 0 ? (int)blockIdx.x : tile);
  const int* s = reinterpret_cast<const int*>(gparts + p);
  int* d = reinterpret_cast<int*>(&sm);
  constexpr int nw = sizeof(DPart) / 4;
  for (int t = threadIdx.x; t < nw; t += blockDim.x) d[t] = __ldg(s + t);
  return p;
}

// Part p of a second level, into shared memory.
__device__ __forceinline__ void part_of(const DPart* __restrict__ gparts, int p, DPart& sm) {
  const int* s = reinterpret_cast<const int*>(gparts + p);
  int* d = reinterpret_cast<int*>(&sm);
  constexpr int nw = sizeof(DPart) / 4;
  for (int t = threadIdx.x; t < nw; t += blockDim.x) d[t] = __ldg(s + t);
}

// Copy one part descriptor into shared memory (all threads of the block call).
__device__ __forceinline__ void stage_part(DPart& dst, const DPart* __restrict__ src) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(&dst);
  constexpr int nw = sizeof(DPart) / 4;
  for (int t = threadIdx.x; t < nw; t += blockDim.x) d[t] = __ldg(s + t);
}

__device__ __forceinline__ void cell_coords(const DPart& p, int c, int& i, int& j, int& k) {
  unsigned q = fdiv((unsigned)c, p.dx);
  i = c - (int)q * p.n[0];
  k = (int)fdiv((unsigned)c, p.dxy);
  j = (int)q - k * p.n[1];
}

__device__ __forceinline__ bool inside(const DPart& p, int i, int j, int k) {
  return (unsigned)i < (unsigned)p.n[0] && (unsigned)j < (unsigned)p.n[1] &&
         (unsigned)k < (unsigned)p.n[2];
}

__device__ __forceinline__ double coef_at(const DPart& p, const double* __restrict__ coef, int e,
                                          int c) {
  long long o = p.coef[e];
  return o >= 0 ? coef[o + c] : p.cval[e];
}
__device__ __forceinline__ float coef_at(const DPart& p, const float* __restrict__ coef, int e,
                                         int c) {
  long long o = p.coef[e];
  return o >= 0 ? coef[o + c] : p.cval32[e];
}

// (S x)(c) for local cell c = (i, j, k) of part p; x points at the level
// vector.  The entry count is uniform over a block, so the dispatch below does
// not diverge.  Fully unrolled variants (7, 15 and 27 entries) issue all loads
// of a cell together.  Parts whose entries are all per cell (every coarse
// level) address entry e as a[e * ncell]; the full 27-point stencil in
// offset-code order derives offsets and bounds from e at compile time.
template <class T>
__device__ __forceinline__ T const_of(const DPart& p, int e);
template <>
__device__ __forceinline__ double const_of<double>(const DPart& p, int e) { return p.cval[e]; }
template <>
__device__ __forceinline__ float const_of<float>(const DPart& p, int e) { return p.cval32[e]; }

template <class T>
__device__ __forceinline__ T stencil27_canon(const DPart& p, const T* __restrict__ a,
                                             const T* __restrict__ xc, int i, int j, int k,
                                             bool interior) {
  const int nx = p.n[0], nxy = p.n[0] * p.n[1], s = p.ncell;
  const bool xm = i > 0, xp = i < p.n[0] - 1, ym = j > 0, yp = j < p.n[1] - 1, zm = k > 0,
             zp = k < p.n[2] - 1;
  T acc = (T)0;
#pragma unroll
  for (int e = 0; e < 27; ++e) {
    const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
    const bool ok = interior || ((dx == 0 || (dx < 0 ? xm : xp)) && (dy == 0 || (dy < 0 ? ym : yp)) &&
                                 (dz == 0 || (dz < 0 ? zm : zp)));
    if (ok) acc = fma(a[e * s], xc[dx + dy * nx + dz * nxy], acc);
  }
  return acc;
}

template <int K, class T>
__device__ __forceinline__ T stencil_fixed(const DPart& p, const T* __restrict__ coef,
                                           const T* __restrict__ xc, int c, int i, int j, int k,
                                           bool interior) {
  T acc = (T)0;
  if (p.allvar) {
    const T* a = coef + p.coef[0] + c;
    const int s = p.ncell;
#pragma unroll
    for (int e = 0; e < K; ++e)
      if (interior || inside(p, i + p.o[e][0], j + p.o[e][1], k + p.o[e][2]))
        acc = fma(a[e * s], xc[p.disp[e]], acc);
  } else {
    const unsigned vm = p.varmask;
#pragma unroll
    for (int e = 0; e < K; ++e)
      if (interior || inside(p, i + p.o[e][0], j + p.o[e][1], k + p.o[e][2])) {
        const T ae = ((vm >> e) & 1u) ? coef[p.coef[e] + c] : const_of<T>(p, e);
        acc = fma(ae, xc[p.disp[e]], acc);
      }
  }
  return acc;
}

// Unchecked form: every entry per cell and zero where it leaves the box, and x
// readable (finite) one plane beyond each end of the level vector, so every
// cell takes the same path with no bounds tests.
template <int K, class T>
__device__ __forceinline__ T stencil_unchecked(const DPart& p, const T* __restrict__ a,
                                               const T* __restrict__ xc) {
  const int s = p.ncell;
  T acc = (T)0;
#pragma unroll
  for (int e = 0; e < K; ++e) acc = fma(a[e * s], xc[p.disp[e]], acc);
  return acc;
}

template <class T>
__device__ __forceinline__ T stencil27_unchecked(const DPart& p, const T* __restrict__ a,
                                                 const T* __restrict__ xc) {
  const int nx = p.n[0], nxy = p.n[0] * p.n[1], s = p.ncell;
  T acc = (T)0;
#pragma unroll
  for (int e = 0; e < 27; ++e) {
    const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
    acc = fma(a[e * s], xc[dx + dy * nx + dz * nxy], acc);
  }
  return acc;
}

template <class T>
__device__ __forceinline__ T stencil_apply(const DPart& p, const T* __restrict__ coef,
                                           const T* __restrict__ x, int c, int i, int j, int k,
                                           bool interior, bool padded) {
  const T* xc = x + p.off + c;
  if (p.allvar && p.zeroext && padded) {
    const T* a = coef + p.coef[0] + c;
    if (p.canon27) return stencil27_unchecked(p, a, xc);
    switch (p.nent) {
      case 7: return stencil_unchecked<7>(p, a, xc);
      case 15: return stencil_unchecked<15>(p, a, xc);
      case 27: return stencil_unchecked<27>(p, a, xc);
      default: break;
    }
  }
  if (p.canon27 && p.allvar) return stencil27_canon(p, coef + p.coef[0] + c, xc, i, j, k, interior);
  switch (p.nent) {
    case 7: return stencil_fixed<7>(p, coef, xc, c, i, j, k, interior);
    case 15: return stencil_fixed<15>(p, coef, xc, c, i, j, k, interior);
    case 27: return stencil_fixed<27>(p, coef, xc, c, i, j, k, interior);
    default: break;
  }
  T acc = (T)0;
#pragma unroll 4
  for (int e = 0; e < p.nent; ++e)
    if (interior || inside(p, i + p.o[e][0], j + p.o[e][1], k + p.o[e][2]))
      acc = fma(coef_at(p, coef, e, c), xc[p.disp[e]], acc);
  return acc;
}

// ---------------------------------------------------------------------------
// Shape-specialised operator apply.  The host picks one shape per level so a
// kernel instance contains only the variant it runs (small code, no per-part
// dispatch).  Unchecked shapes need every entry per cell, zero outside the
// box, and a guard-padded x; the checked shape handles constant entries and
// caller vectors with branch-free bounds handling (an out-of-box neighbour
// reads the cell itself and is multiplied by zero).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_interior(const DPart& p, int i, int j, int k) {
  return i > 0 && i < p.n[0] - 1 && j > 0 && j < p.n[1] - 1 && k > 0 && k < p.n[2] - 1;
}

enum StencilShape { SH_CHECKED = 0, SH_U7 = 1, SH_U15 = 2, SH_C27 = 3, SH_UGEN = 4, SH_K7 = 5 };

// Checked 7-point stencil in the canonical entry order (centre, -x, +x, -y,
// +y, -z, +z): directions and bounds are known at compile time; entries may
// be constant or per cell (uniform per part).
template <class T>
__device__ __forceinline__ T stencil7_canon_checked(const DPart& p, const T* __restrict__ coef,
                                                    const T* __restrict__ xc, int c, int i, int j,
                                                    int k) {
  const int nx = p.n[0], nxy = p.n[0] * p.n[1];
  const bool ok[7] = {true, i > 0, i < p.n[0] - 1, j > 0, j < p.n[1] - 1, k > 0, k < p.n[2] - 1};
  const int d[7] = {0, -1, 1, -nx, nx, -nxy, nxy};
  const unsigned vm = p.varmask;
  T acc = (T)0;
#pragma unroll
  for (int e = 0; e < 7; ++e) {
    const T ae = ((vm >> e) & 1u) ? coef[p.coef[e] + c] : const_of<T>(p, e);
    const T xv = xc[ok[e] ? d[e] : 0];
    acc = fma(ae, ok[e] ? xv : (T)0, acc);
  }
  return acc;
}

template <int K, class T>
__device__ __forceinline__ T stencil_checked_fixed(const DPart& p, const T* __restrict__ coef,
                                                   const T* __restrict__ xc, int c, int i, int j,
                                                   int k) {
  const bool xm = i > 0, xp = i < p.n[0] - 1, ym = j > 0, yp = j < p.n[1] - 1, zm = k > 0,
             zp = k < p.n[2] - 1;
  const unsigned vm = p.varmask;
  T acc = (T)0;
#pragma unroll
  for (int e = 0; e < K; ++e) {
    const int ox = p.o[e][0], oy = p.o[e][1], oz = p.o[e][2];
    const bool ok = (ox == 0 || (ox < 0 ? xm : xp)) && (oy == 0 || (oy < 0 ? ym : yp)) &&
                    (oz == 0 || (oz < 0 ? zm : zp));
    const T ae = ((vm >> e) & 1u) ? coef[p.coef[e] + c] : const_of<T>(p, e);
    const T xv = xc[ok ? p.disp[e] : 0];
    acc = fma(ae, ok ? xv : (T)0, acc);
  }
  return acc;
}

template <class T>
__device__ __forceinline__ T stencil_checked_loop(const DPart& p, const T* __restrict__ coef,
                                                  const T* __restrict__ xc, int c, int i, int j,
                                                  int k) {
  T acc = (T)0;
#pragma unroll 4
  for (int e = 0; e < p.nent; ++e) {
    const bool ok = inside(p, i + p.o[e][0], j + p.o[e][1], k + p.o[e][2]);
    const T xv = xc[ok ? p.disp[e] : 0];
    acc = fma(coef_at(p, coef, e, c), ok ? xv : (T)0, acc);
  }
  return acc;
}

template <int SH, class T>
__device__ __forceinline__ T stencil_sh(const DPart& p, const T* __restrict__ coef,
                                        const T* __restrict__ x, int c, int i, int j, int k) {
  const T* xc = x + p.off + c;
  if constexpr (SH == SH_C27) {
    return stencil27_unchecked(p, coef + p.coef[0] + c, xc);
  } else if constexpr (SH == SH_U7) {
    return stencil_unchecked<7>(p, coef + p.coef[0] + c, xc);
  } else if constexpr (SH == SH_U15) {
    return stencil_unchecked<15>(p, coef + p.coef[0] + c, xc);
  } else if constexpr (SH == SH_K7) {
    return stencil7_canon_checked(p, coef, xc, c, i, j, k);
  } else if constexpr (SH == SH_UGEN) {
    // parts of one level with different stencils (e.g. semicoarsened in
    // different directions): the unrolled form of each part's size, chosen
    // per part (uniform over a block), so that every entry's loads are in
    // flight together; the same entry order as a plain loop
    const T* a = coef + p.coef[0] + c;
    if (p.canon27) return stencil27_unchecked(p, a, xc);
    if (p.nent == 15) return stencil_unchecked<15>(p, a, xc);
    if (p.nent == 7) return stencil_unchecked<7>(p, a, xc);
    const int s = p.ncell, n = p.nent;
    T acc = (T)0;
#pragma unroll
    for (int e = 0; e < SSAMG_MAXE; ++e)
      if (e < n) acc = fma(a[e * s], xc[p.disp[e]], acc);
    return acc;
  } else {
    if (p.nent == 7) return stencil_checked_fixed<7>(p, coef, xc, c, i, j, k);
    return stencil_checked_loop(p, coef, xc, c, i, j, k);
  }
}

// (A x)(g) for local cell c of part p with shape SH; coordinates are only
// computed where needed (checked shape, or face cells of coupled parts).
// has_u: 1 = the part's coupling rows lie on its box faces, 2 = anywhere
// (rows inside the box, e.g. beside ghost unknowns), so every cell adds U x.
template <int SH, class T>
__device__ __forceinline__ T apply_A_sh(const LevelView<T>& L, const DPart& p,
                                        const T* __restrict__ x, int c) {
  int i = 0, j = 0, k = 0;
  if (SH == SH_CHECKED || SH == SH_K7 || p.has_u) cell_coords(p, c, i, j, k);
  T acc = stencil_sh<SH>(p, L.coef, x, c, i, j, k);
  if (p.has_u > 1 || (p.has_u && !is_interior(p, i, j, k))) acc += L.uy[p.off + c];
  return acc;
}

// The unchecked shapes for R right-hand sides at once: each stencil
// coefficient is loaded once and multiplies the R vectors' neighbours (x of
// right-hand side q at x + q vs); each right-hand side's sum takes the
// entries in the single form's order, so acc[q] is bitwise what
// stencil_sh gives for x + q vs.
template <int K, int R, class T>
__device__ __forceinline__ void stencil_unchecked_r(const DPart& p, const T* __restrict__ a,
                                                    const T* __restrict__ xc, long long vs,
                                                    T* acc) {
  const int s = p.ncell;
#pragma unroll
  for (int q = 0; q < R; ++q) acc[q] = (T)0;
#pragma unroll
  for (int e = 0; e < K; ++e) {
    const T ae = a[e * s];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] = fma(ae, xc[q * vs + p.disp[e]], acc[q]);
  }
}

template <int R, class T>
__device__ __forceinline__ void stencil27_unchecked_r(const DPart& p, const T* __restrict__ a,
                                                      const T* __restrict__ xc, long long vs,
                                                      T* acc) {
  const int nx = p.n[0], nxy = p.n[0] * p.n[1], s = p.ncell;
#pragma unroll
  for (int q = 0; q < R; ++q) acc[q] = (T)0;
#pragma unroll
  for (int e = 0; e < 27; ++e) {
    const int dx = e % 3 - 1, dy = (e / 3) % 3 - 1, dz = e / 9 - 1;
    const T ae = a[e * s];
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] = fma(ae, xc[q * vs + dx + dy * nx + dz * nxy], acc[q]);
  }
}

// Shapes with a several-right-hand-side form: every entry per cell.
__host__ __device__ constexpr bool shape_has_rhs_form(int sh) {
  return sh == SH_U7 || sh == SH_U15 || sh == SH_C27 || sh == SH_UGEN;
}

template <int SH, int R, class T>
__device__ __forceinline__ void stencil_sh_r(const DPart& p, const T* __restrict__ coef,
                                             const T* __restrict__ x, int c, long long vs,
                                             T* acc) {
  const T* xc = x + p.off + c;
  const T* a = coef + p.coef[0] + c;
  if constexpr (SH == SH_C27) {
    stencil27_unchecked_r<R>(p, a, xc, vs, acc);
  } else if constexpr (SH == SH_U7) {
    stencil_unchecked_r<7, R>(p, a, xc, vs, acc);
  } else if constexpr (SH == SH_U15) {
    stencil_unchecked_r<15, R>(p, a, xc, vs, acc);
  } else {
    static_assert(SH == SH_UGEN, "no several-right-hand-side form of this shape");
    if (p.canon27) {
      stencil27_unchecked_r<R>(p, a, xc, vs, acc);
    } else if (p.nent == 15) {
      stencil_unchecked_r<15, R>(p, a, xc, vs, acc);
    } else if (p.nent == 7) {
      stencil_unchecked_r<7, R>(p, a, xc, vs, acc);
    } else {
      const int s = p.ncell, n = p.nent;
#pragma unroll
      for (int q = 0; q < R; ++q) acc[q] = (T)0;
#pragma unroll
      for (int e = 0; e < SSAMG_MAXE; ++e)
        if (e < n) {
          const T ae = a[e * s];
#pragma unroll
          for (int q = 0; q < R; ++q) acc[q] = fma(ae, xc[q * vs + p.disp[e]], acc[q]);
        }
    }
  }
}

// (A x_q)(c) for R right-hand sides (x_q = x + q vs, U x_q likewise in uy),
// each bitwise apply_A_sh's value.
template <int SH, int R, class T>
__device__ __forceinline__ void apply_A_sh_r(const LevelView<T>& L, const DPart& p,
                                             const T* __restrict__ x, int c, long long vs,
                                             T* acc) {
  int i = 0, j = 0, k = 0;
  if (p.has_u) cell_coords(p, c, i, j, k);
  stencil_sh_r<SH, R>(p, L.coef, x, c, vs, acc);
  if (p.has_u > 1 || (p.has_u && !is_interior(p, i, j, k))) {
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] += L.uy[p.off + c + q * vs];
  }
}

// (U x)(g) for global cell g (0 when g has no U row).
template <class T>
__device__ __forceinline__ T u_apply(const LevelView<T>& L, const T* __restrict__ x, int g) {
  int r = __ldg(L.u_map + g);
  T acc = (T)0;
  if (r >= 0) {
    int q1 = __ldg(L.u_ptr + r + 1);
    for (int q = __ldg(L.u_ptr + r); q < q1; ++q) acc = fma(L.u_val[q], x[__ldg(L.u_col + q)], acc);
  }
  return acc;
}


// (A x)(c) = (S x)(c) + (U x)(c); the U part comes from L.uy, which a row
// job filled for this same x (only face cells can have couplings unless
// has_u is 2).
template <class T>
__device__ __forceinline__ T apply_A(const LevelView<T>& L, const DPart& p, const T* __restrict__ x,
                                     int c, int i, int j, int k, bool padded = true) {
  bool interior = is_interior(p, i, j, k);
  T acc = stencil_apply(p, L.coef, x, c, i, j, k, interior, padded);
  if (p.has_u > 1 || (p.has_u && !interior)) acc += L.uy[p.off + c];
  return acc;
}

// Sum of one U row: the L.tpr lanes l4 of a row group compute
// sum_q u_q * f(col_q, q, s_q) for row r (r >= L.nr: nothing, but the lanes
// still join the shuffles) and store it at the row's cell of L.uy;
// s_q = pre(col_q, q) is the entry's setup-time data.  With WAIT, the row
// bounds, each lane's first column and value, and pre() of that entry are
// loaded before pdl_wait(); so a row of at most L.tpr entries (the level
// picks tpr from its mean row length) has one dependent load after the
// wait.  pre() may read only what setup wrote.  Further entries go four per
// lane at a time so that their loads overlap; the summation order is that
// of q ascending per lane, then a fixed shuffle tree over the lanes.
template <bool WAIT, class T, class Pre, class F>
__device__ __forceinline__ void u_row_sum(const LevelView<T>& L, int r, int l4, Pre&& pre,
                                          F&& f) {
  const int tp = L.tpr;
  int q = 0, q1 = 0, c0 = 0;
  T u0 = (T)0;
  decltype(pre(0, 0)) s0{};
  if (r < L.nr) {
    q = L.u_ptr[r] + l4;
    q1 = L.u_ptr[r + 1];
    if (q < q1) {
      c0 = L.u_col[q];
      u0 = L.u_val[q];
      s0 = pre(c0, q);
    }
  }
  if constexpr (WAIT) pdl_wait();
  T acc = (T)0;
  if (q < q1) {
    acc = fma(u0, f(c0, q, s0), acc);
    q += tp;
    for (; q + 3 * tp < q1; q += 4 * tp) {
      const int c1 = L.u_col[q], c2 = L.u_col[q + tp], c3 = L.u_col[q + 2 * tp],
                c4 = L.u_col[q + 3 * tp];
      const T u1 = L.u_val[q], u2 = L.u_val[q + tp], u3 = L.u_val[q + 2 * tp],
              u4 = L.u_val[q + 3 * tp];
      const T v1 = f(c1, q, pre(c1, q)), v2 = f(c2, q + tp, pre(c2, q + tp)),
              v3 = f(c3, q + 2 * tp, pre(c3, q + 2 * tp)),
              v4 = f(c4, q + 3 * tp, pre(c4, q + 3 * tp));
      acc = fma(u1, v1, acc);
      acc = fma(u2, v2, acc);
      acc = fma(u3, v3, acc);
      acc = fma(u4, v4, acc);
    }
    for (; q < q1; q += tp) {
      const int c = L.u_col[q];
      acc = fma(L.u_val[q], f(c, q, pre(c, q)), acc);
    }
  }
  for (int o = 1; o < tp; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (r < L.nr && l4 == 0) L.uy[L.u_rows[r]] = acc;
}

// Row job of a launch: block rb's threads take SSAMG_BLOCK / L.tpr rows,
// L.tpr lanes each (all threads must call; waits for the predecessor inside).
template <class T, class Pre, class F>
__device__ __forceinline__ void u_row_job(const LevelView<T>& L, int rb, Pre&& pre, F&& f) {
  const int sh = __ffs(L.tpr) - 1;  // tpr is a power of two
  u_row_sum<true>(L, rb * (SSAMG_BLOCK >> sh) + ((int)threadIdx.x >> sh),
                  (int)threadIdx.x & (L.tpr - 1), pre, f);
}

// Block-wide sum (deterministic: fixed order).  sh holds NT doubles.  The
// threads' values go through shared memory and one warp adds them: lane l
// sums values l, l + 32, ... in order, then a fixed shuffle tree.  FP64 adds
// run at 1/64 of the FP32 rate on this GPU, so a shuffle tree in every warp
// (5 adds per thread) cost as much as the kernels' own FP64 work when each
// thread holds a few cells; this takes NT/32 - 1 + 5 adds in one warp.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = sh[threadIdx.x];
#pragma unroll
    for (int q = 1; q < NT / 32; ++q) r += sh[threadIdx.x + 32 * q];
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// Fine-point index (within the part's P arrays) of local fine cell (i, j, k).
__device__ __forceinline__ int fine_point_index(const DPart& p, int i, int j, int k) {
  // selects rather than an array indexed by d* (which would live in local memory)
  const int d = p.dstar;
  if (d == 0)
    i = (i + p.par) >> 1;
  else if (d == 1)
    j = (j + p.par) >> 1;
  else
    k = (k + p.par) >> 1;
  return (k * p.nf[1] + j) * p.nf[0] + i;
}

// Linear index on the next level of local coarse cell (i, j, k).
__device__ __forceinline__ int coarse_index(const DPart& p, int i, int j, int k) {
  return p.coff + (k * p.cn[1] + j) * p.cn[0] + i;
}

// P's row for local fine cell (i, j, k) of part p (Section 3.2): a coarse
// point maps to itself with weight 1; a fine point to its west and east
// coarse neighbours along d* (when inside the box) with PW, PE.  Columns are
// coarse-level indices, -1 where absent; j0 is the west (or only) one.
template <class T>
struct PRow {
  int j0, j1;
  T w0, w1;
};

template <class T>
__device__ __forceinline__ PRow<T> p_row(const DPart& p, const T* __restrict__ Pw,
                                         const T* __restrict__ Pe, int i, int j, int k) {
  PRow<T> r{-1, -1, (T)0, (T)0};
  const int d = p.dstar;
  if (d < 0) {
    r.j0 = coarse_index(p, i, j, k);
    r.w0 = (T)1;
    return r;
  }
  // coarse index of (i, j, k) with its d* component replaced by v (selects,
  // not an array indexed by d*)
  auto at = [&](int v) {
    return coarse_index(p, d == 0 ? v : i, d == 1 ? v : j, d == 2 ? v : k);
  };
  const int cd = d == 0 ? i : (d == 1 ? j : k);
  if (((cd + p.par) & 1) == 0) {
    r.j0 = at((cd - p.par) >> 1);
    r.w0 = (T)1;
    return r;
  }
  const int F = p.poff + fine_point_index(p, i, j, k);
  if (cd - 1 >= 0) {
    r.j0 = at((cd - 1 - p.par) >> 1);
    r.w0 = Pw[F];
  }
  if (cd + 1 < p.n[d]) {
    r.j1 = at((cd + 1 - p.par) >> 1);
    r.w1 = Pe[F];
  }
  if (r.j0 < 0) {  // only the east neighbour: keep it first
    r.j0 = r.j1;
    r.w0 = r.w1;
    r.j1 = -1;
    r.w1 = (T)0;
  }
  return r;
}

// x + P e at one fine cell: the row's terms added west first, as the
// oracle's P^T / P pair orders them.
template <class T>
__device__ __forceinline__ T add_p_row(T v, const PRow<T>& r, const T* __restrict__ ec) {
  if (r.j0 >= 0) v = fma(r.w0, ec[r.j0], v);
  if (r.j1 >= 0) v = fma(r.w1, ec[r.j1], v);
  return v;
}
