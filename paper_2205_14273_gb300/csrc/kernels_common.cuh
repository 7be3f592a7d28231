// Device helpers shared by the kernel translation units.
#pragma once

#include "ssamg_internal.cuh"

// Cell-wise launches give each block a tile of SSAMG_TILE consecutive cells of
// one part; thread t handles cells t, t + SSAMG_BLOCK, ... (coalesced), so
// per-block work (descriptor staging, reductions) is amortised over
// SSAMG_CPT cells per thread.
#define TILE_LOOP(c, first, count)                                                         \
  for (int c##_m = 0, c = ((int)blockIdx.x - (first)) * SSAMG_TILE + (int)threadIdx.x;     \
       c##_m < SSAMG_CPT && c < (count); ++c##_m, c += SSAMG_BLOCK)

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

// (S x)(c) for local cell c = (i, j, k) of part p; x points at the level vector.
template <class T>
__device__ __forceinline__ T stencil_apply(const DPart& p, const T* __restrict__ coef,
                                           const T* __restrict__ x, int c, int i, int j, int k,
                                           bool interior) {
  const T* xc = x + p.off + c;
  T acc = (T)0;
  if (interior) {
    for (int e = 0; e < p.nent; ++e) acc = fma(coef_at(p, coef, e, c), xc[p.disp[e]], acc);
  } else {
    for (int e = 0; e < p.nent; ++e) {
      if (inside(p, i + p.o[e][0], j + p.o[e][1], k + p.o[e][2]))
        acc = fma(coef_at(p, coef, e, c), xc[p.disp[e]], acc);
    }
  }
  return acc;
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

__device__ __forceinline__ bool is_interior(const DPart& p, int i, int j, int k) {
  return i > 0 && i < p.n[0] - 1 && j > 0 && j < p.n[1] - 1 && k > 0 && k < p.n[2] - 1;
}

// (A x)(c) = (S x + U x)(c).
template <class T>
__device__ __forceinline__ T apply_A(const LevelView<T>& L, const DPart& p, const T* __restrict__ x,
                                     int c, int i, int j, int k) {
  bool interior = is_interior(p, i, j, k);
  T acc = stencil_apply(p, L.coef, x, c, i, j, k, interior);
  if (p.has_u && !interior) acc += u_apply(L, x, p.off + c);
  return acc;
}

// Block-wide sum (deterministic: fixed shuffle tree, then fixed warp order).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (l < NT / 32) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;  // valid in thread 0
}

// Fine-point index (within the part's P arrays) of local fine cell (i, j, k).
__device__ __forceinline__ int fine_point_index(const DPart& p, int i, int j, int k) {
  int c[3] = {i, j, k};
  c[p.dstar] = (c[p.dstar] + p.par) >> 1;
  return (c[2] * p.nf[1] + c[1]) * p.nf[0] + c[0];
}

// Linear index on the next level of local coarse cell (i, j, k).
__device__ __forceinline__ int coarse_index(const DPart& p, int i, int j, int k) {
  return p.coff + (k * p.cn[1] + j) * p.cn[0] + i;
}

// Columns of P's row for local fine cell (i, j, k) of part p (Section 3.2):
// a coarse point maps to itself with weight 1; a fine point to its west and
// east coarse neighbours along d* (when inside the box) with PW, PE.
template <class T>
__device__ __forceinline__ int p_row(const DPart& p, const T* __restrict__ Pw,
                                     const T* __restrict__ Pe, int i, int j, int k, int* J, T* w) {
  if (p.dstar < 0) {
    J[0] = coarse_index(p, i, j, k);
    w[0] = (T)1;
    return 1;
  }
  int c[3] = {i, j, k};
  const int d = p.dstar;
  const int cd = c[d];
  if (((cd + p.par) & 1) == 0) {
    c[d] = (cd - p.par) >> 1;
    J[0] = coarse_index(p, c[0], c[1], c[2]);
    w[0] = (T)1;
    return 1;
  }
  int F = p.poff + fine_point_index(p, i, j, k);
  int m = 0;
  if (cd - 1 >= 0) {
    c[d] = (cd - 1 - p.par) >> 1;
    J[m] = coarse_index(p, c[0], c[1], c[2]);
    w[m++] = Pw[F];
  }
  if (cd + 1 < p.n[d]) {
    c[d] = (cd + 1 - p.par) >> 1;
    J[m] = coarse_index(p, c[0], c[1], c[2]);
    w[m++] = Pe[F];
  }
  return m;
}
