// Coarse-level transition (the hybrid idea of Section 3.5): below a chosen
// level the V-cycle leaves the stencil kernels.  At setup every level from
// the transition level T down to the coarsest is assembled: A_l = S_l + U_l
// as CSR rows (stencil entries inside the box in entry order, then the
// couplings), the smoother diagonal omega M^-1 (Section 3.4), P's row of
// every fine cell (Section 3.2) and the restriction row P^T of every coarse
// cell, and the coarsest operator's explicit inverse.  The rows of each level
// are split into NC contiguous slices, one per CTA of a thread-block cluster;
// each CTA's share is laid out as one contiguous image in global memory.
//
// In the solve one cluster runs the whole tail of the V(1,1) cycle: every
// CTA copies its image into shared memory, the level vectors (x, b, r) live
// in the CTAs' shared memory (distributed shared memory: a column index packs
// the owning CTA and the position in its slice), and cluster barriers
// separate the steps that other launches separate elsewhere: pre-relaxation
// from zero, residual, restriction, coarsest solve, prolongation, post-
// relaxation (Eq. relax0).  Every row is summed in a fixed order (its
// entries strided over a group of lanes, then a fixed shuffle tree), so a tail
// result is the same bit for bit from run to run.
#include <cooperative_groups.h>

#include <map>
#include <mutex>
#include <tuple>

#include "kernels_common.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int CT = SSAMG_CTAIL_THREADS;

// Packed column: owning CTA (high bits) and position in its slice.
__device__ __forceinline__ unsigned short ctail_pack(int g, int S) {
  const int o = g / S;
  return (unsigned short)((o << SSAMG_CTAIL_LOCAL_BITS) | (g - o * S));
}

// Row lengths of the tail levels: entries of S inside the box plus the row's
// couplings.
// Row lengths of one level, a warp per row: lane e tests entry e.
__device__ __forceinline__ void ctail_rowlen_row(const LevelView<double>& L, int* __restrict__ len,
                                                 int g) {
  const int lane = threadIdx.x & 31;
  if (g >= L.N) return;
  const int p = find_part_cell(L.cellstart, L.np, g);
  const DPart& dp = L.parts[p];
  int i, j, k;
  cell_coords(dp, g - dp.off, i, j, k);
  const bool ok = lane < dp.nent && inside(dp, i + dp.o[lane][0], j + dp.o[lane][1], k + dp.o[lane][2]);
  int n = __popc(__ballot_sync(0xffffffffu, ok));
  if (lane == 0) {
    if (dp.has_u && L.u_map) {
      const int r = L.u_map[g];
      if (r >= 0) n += L.u_ptr[r + 1] - L.u_ptr[r];
    }
    len[g] = n;
  }
}

// Every candidate level in one launch: block b works on the level whose
// block range holds it (8 rows per block).
struct CTailRowlenArgs {
  int nl;
  int b0[SSAMG_CTAIL_MAX_LEVELS + 1];
  int* len[SSAMG_CTAIL_MAX_LEVELS];
  LevelView<double> lv[SSAMG_CTAIL_MAX_LEVELS];
};
__global__ void __launch_bounds__(256) k_ctail_rowlen(const __grid_constant__ CTailRowlenArgs A) {
  int l = 0;
  while (l + 1 < A.nl && (int)blockIdx.x >= A.b0[l + 1]) ++l;
  const int g = ((int)blockIdx.x - A.b0[l]) * 8 + (int)(threadIdx.x >> 5);
  ctail_rowlen_row(A.lv[l], A.len[l], g);
}

// Fills the images of one tail level l: for every row g, in the slice of its
// owning CTA: its CSR entries (columns packed in this level's slices), the
// smoother diagonal, P's row (columns packed in level l+1's slices) when
// has_p, the restriction row from level l-1 (columns packed in l-1's
// slices) when Fm is given, and the coarsest inverse's row when inv is
// given.  The row pointers were written by the host.
// One tail level's share of a fill launch.
struct CTailFillLevel {
  LevelView<double> L, fm, ln;
  const double* dinv;
  const double* inv;
  CTailLevel lv;
  int has_fm, has_p, Sm, Sn;
};
struct CTailFillArgs {
  int nl, nL;
  long long ro_bytes;
  char* image;
  int b0[SSAMG_CTAIL_MAX_LEVELS + 1];
  CTailFillLevel lev[SSAMG_CTAIL_MAX_LEVELS];
};

template <class T>
__device__ __forceinline__ void ctail_fill_row(const LevelView<double>& L,
                                               const double* __restrict__ dinv64,
                                               const LevelView<double>& Fm, int has_fm,
                                               const LevelView<double>& Ln, int has_p,
                                               const double* __restrict__ inv, int nL,
                                               const CTailLevel& lv, int Sm, int Sn,
                                               char* __restrict__ image, long long ro_bytes,
                                               int g) {
  // a warp per row: the stencil entries one per lane (slots by ballot, in
  // entry order), the coupling entries strided over the lanes, the rest by
  // lane 0
  const int lane = threadIdx.x & 31;
  if (g >= L.N) return;
  const int owner = g / lv.S, li = g - owner * lv.S;
  char* img = image + owner * ro_bytes;
  const int* rowptr = reinterpret_cast<const int*>(img + lv.o_rowptr);
  unsigned short* col = reinterpret_cast<unsigned short*>(img + lv.o_col);
  T* val = reinterpret_cast<T*>(img + lv.o_val);
  T* dv = reinterpret_cast<T*>(img + lv.o_dinv);
  const int p = find_part_cell(L.cellstart, L.np, g);
  const DPart& dp = L.parts[p];
  const int c = g - dp.off;
  int i, j, k;
  cell_coords(dp, c, i, j, k);
  const int q0 = rowptr[li];
  const bool ok = lane < dp.nent && inside(dp, i + dp.o[lane][0], j + dp.o[lane][1], k + dp.o[lane][2]);
  const unsigned m = __ballot_sync(0xffffffffu, ok);
  if (ok) {
    const int q = q0 + __popc(m & ((1u << lane) - 1u));
    col[q] = ctail_pack(g + dp.disp[lane], lv.S);
    val[q] = (T)coef_at(dp, L.coef, lane, c);
  }
  if (dp.has_u && L.u_map) {
    const int r = L.u_map[g];
    if (r >= 0) {
      const int t0 = L.u_ptr[r], t1 = L.u_ptr[r + 1], q1 = q0 + __popc(m) - t0;
      for (int t = t0 + lane; t < t1; t += 32) {
        col[q1 + t] = ctail_pack(L.u_col[t], lv.S);
        val[q1 + t] = (T)L.u_val[t];
      }
    }
  }
  if (inv) {
    double* iv = reinterpret_cast<double*>(img + lv.o_inv);
    for (int t = lane; t < nL; t += 32) iv[(long long)li * nL + t] = inv[(long long)g * nL + t];
  }
  if (lane != 0) return;
  dv[li] = (T)dinv64[g];
  if (has_p) {
    // P's row of fine cell g (Section 3.2), coarse columns on level l+1
    const PRow<double> pr = p_row(dp, L.Pw, L.Pe, i, j, k);
    unsigned short* pc = reinterpret_cast<unsigned short*>(img + lv.o_pcol);
    T* pv = reinterpret_cast<T*>(img + lv.o_pval);
    pc[li] = pr.j0 >= 0 ? ctail_pack(pr.j0, Sn) : 0;
    pv[li] = pr.j0 >= 0 ? (T)pr.w0 : (T)0;
    pc[lv.S + li] = pr.j1 >= 0 ? ctail_pack(pr.j1, Sn) : 0;
    pv[lv.S + li] = pr.j1 >= 0 ? (T)pr.w1 : (T)0;
  }
  if (has_fm) {
    // restriction row of coarse cell g from level l-1: the anchor (weight 1)
    // and the fine points beside it along d* (PE of the west one, PW of the
    // east one), as the stencil restriction applies them
    const DPart& fp = Fm.parts[p];
    unsigned short* rc = reinterpret_cast<unsigned short*>(img + lv.o_rcol);
    T* rv = reinterpret_cast<T*>(img + lv.o_rval);
    int f0, f1 = -1, f2 = -1;
    double w1 = 0.0, w2 = 0.0;
    const int d = fp.dstar;
    if (d < 0) {
      f0 = fp.off + (k * fp.n[1] + j) * fp.n[0] + i;
    } else {
      int f[3] = {i, j, k};
      const int anchor = 2 * f[d] + fp.par;
      f[d] = anchor;
      const int sd = (d == 0) ? 1 : (d == 1 ? fp.n[0] : fp.n[0] * fp.n[1]);
      f0 = fp.off + (f[2] * fp.n[1] + f[1]) * fp.n[0] + f[0];
      if (anchor - 1 >= 0) {
        f[d] = anchor - 1;
        f1 = f0 - sd;
        w1 = Fm.Pe[fp.poff + fine_point_index(fp, f[0], f[1], f[2])];
      }
      if (anchor + 1 < fp.n[d]) {
        f[d] = anchor + 1;
        f2 = f0 + sd;
        w2 = Fm.Pw[fp.poff + fine_point_index(fp, f[0], f[1], f[2])];
      }
    }
    rc[li] = ctail_pack(f0, Sm);
    rv[li] = (T)1;
    rc[lv.S + li] = f1 >= 0 ? ctail_pack(f1, Sm) : 0;
    rv[lv.S + li] = f1 >= 0 ? (T)w1 : (T)0;
    rc[2 * lv.S + li] = f2 >= 0 ? ctail_pack(f2, Sm) : 0;
    rv[2 * lv.S + li] = f2 >= 0 ? (T)w2 : (T)0;
  }
}

// Every tail level's images in one launch (8 rows per block).
template <class T>
__global__ void __launch_bounds__(256) k_ctail_fill(const __grid_constant__ CTailFillArgs A) {
  int l = 0;
  while (l + 1 < A.nl && (int)blockIdx.x >= A.b0[l + 1]) ++l;
  const CTailFillLevel& v = A.lev[l];
  const int g = ((int)blockIdx.x - A.b0[l]) * 8 + (int)(threadIdx.x >> 5);
  ctail_fill_row<T>(v.L, v.dinv, v.fm, v.has_fm, v.ln, v.has_p, v.inv, A.nL, v.lv, v.Sm, v.Sn,
                    A.image, A.ro_bytes, g);
}

// Cluster-wide barrier between the tail's steps.  The non-aligned forms of
// barrier.cluster (release on arrival, acquire on the wait) do not need the
// warp's lanes to arrive together, so a warp whose lanes left a row loop at
// different times still counts as arrived only once every lane has; the
// release/acquire pair makes each CTA's shared-memory writes before the
// barrier visible to every CTA's reads after it.
__device__ __forceinline__ void ctail_sync() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// Value of a packed column of vector `off` (byte offset of that level's
// vector in every CTA's shared memory).
template <class T>
__device__ __forceinline__ T ctail_get(cg::cluster_group& cl, char* sm, int off,
                                       unsigned short pk) {
  const unsigned o = pk >> SSAMG_CTAIL_LOCAL_BITS;
  const unsigned l = pk & ((1u << SSAMG_CTAIL_LOCAL_BITS) - 1u);
  const T* base = cl.map_shared_rank(reinterpret_cast<T*>(sm + off), o);
  return base[l];
}

// Operator apply over the CSR rows of one level's slice: L.tpr lanes take a
// row (its entries strided over the lanes, each lane fetching up to eight of
// its entries before summing them, so that a row's remote loads are in
// flight together), their partial sums are added by a fixed shuffle tree,
// and the row's first lane hands the result to epi(li, (A x)(li)).  The loop
// bound is uniform over each warp, so every lane takes part in the shuffles.
template <class T, class Epi>
__device__ __forceinline__ void ctail_apply(cg::cluster_group& cl, char* sm, int xoff,
                                            const CTailLevel& L, const int* rp,
                                            const unsigned short* col, const T* val, Epi&& epi) {
  const int tpr = L.tpr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int rpw = 32 / tpr;  // rows per warp and pass
  const int sub = lane / tpr, k = lane & (tpr - 1);
  for (int r0 = warp * rpw; r0 < L.S; r0 += (CT / 32) * rpw) {
    const int li = r0 + sub;
    T acc = (T)0;
    if (li < L.S) {
      // this lane's entries q0 + k, q0 + k + tpr, ... eight loads at a time
      const int q1 = rp[li + 1];
      for (int q = rp[li] + k; q < q1; q += 8 * tpr) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          v[u] = q + u * tpr < q1 ? ctail_get<T>(cl, sm, xoff, col[q + u * tpr]) : (T)0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (q + u * tpr < q1) acc = fma(val[q + u * tpr], v[u], acc);
      }
    }
    for (int o = tpr >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (li < L.S && k == 0) epi(li, acc);
  }
}

// The tail of one V(1,1) cycle: from the right-hand side of level T (global,
// b_top) to the corrected x of level T (global, x_top).
template <class T>
__global__ void __launch_bounds__(CT, 1) k_ctail(const CTailArgs a, const T* b_top, T* x_top) {
  pdl_trigger();
  extern __shared__ __align__(16) char sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int c = (int)cl.block_rank();
  const int tid = threadIdx.x;
  // the read-only image (setup data) first, then the wait for the
  // predecessor that wrote b_top
  {
    const int4* src = reinterpret_cast<const int4*>(a.image + (long long)c * a.ro_bytes);
    int4* dst = reinterpret_cast<int4*>(sm + a.vec_bytes);
    const long long n16 = a.ro_bytes / 16;
    for (long long t = tid; t < n16; t += CT) dst[t] = src[t];
  }
  pdl_wait();
  __syncthreads();  // the image (read below: level T's diagonal) is staged
  const int nt = a.nt;
  {
    const CTailLevel& L = a.lev[0];
    T* b = reinterpret_cast<T*>(sm + L.o_b);
    T* x = reinterpret_cast<T*>(sm + L.o_x);
    const T* dv = reinterpret_cast<const T*>(sm + a.vec_bytes + L.o_dinv);
    for (int li = tid; li < L.S; li += CT) {
      const int g = c * L.S + li;
      const T v = g < L.n ? b_top[g] : (T)0;
      b[li] = v;
      x[li] = dv[li] * v;  // pre-relaxation from zero
    }
  }
  // down: residual, then restriction with the coarse level's pre-relaxation
  for (int l = 0; l + 1 < nt; ++l) {
    const CTailLevel& L = a.lev[l];
    const CTailLevel& C = a.lev[l + 1];
    const char* ro = sm + a.vec_bytes;
    const int* rp = reinterpret_cast<const int*>(ro + L.o_rowptr);
    const unsigned short* col = reinterpret_cast<const unsigned short*>(ro + L.o_col);
    const T* val = reinterpret_cast<const T*>(ro + L.o_val);
    const T* b = reinterpret_cast<const T*>(sm + L.o_b);
    T* r = reinterpret_cast<T*>(sm + L.o_r);
    ctail_sync();  // x of level l complete in every CTA
    ctail_apply<T>(cl, sm, L.o_x, L, rp, col, val, [&](int li, T ax) { r[li] = b[li] - ax; });
    ctail_sync();  // r of level l complete
    const unsigned short* rc = reinterpret_cast<const unsigned short*>(ro + C.o_rcol);
    const T* rv = reinterpret_cast<const T*>(ro + C.o_rval);
    const T* dvc = reinterpret_cast<const T*>(ro + C.o_dinv);
    T* bc = reinterpret_cast<T*>(sm + C.o_b);
    T* xc = reinterpret_cast<T*>(sm + C.o_x);
    for (int li = tid; li < C.S; li += CT) {
      T v = rv[li] * ctail_get<T>(cl, sm, L.o_r, rc[li]);
      v = fma(rv[C.S + li], ctail_get<T>(cl, sm, L.o_r, rc[C.S + li]), v);
      v = fma(rv[2 * C.S + li], ctail_get<T>(cl, sm, L.o_r, rc[2 * C.S + li]), v);
      bc[li] = v;
      xc[li] = dvc[li] * v;
    }
  }
  // coarsest level: the dense inverse (FP64) or one relaxation sweep
  {
    const CTailLevel& L = a.lev[nt - 1];
    T* x = reinterpret_cast<T*>(sm + L.o_x);
    if (a.direct) {
      ctail_sync();  // b of the coarsest level complete
      const double* iv = reinterpret_cast<const double*>(sm + a.vec_bytes + L.o_inv);
      for (int li = tid; li < L.S; li += CT) {
        double s = 0.0;
        if (c * L.S + li < L.n) {
          int t = 0;
          for (; t + 8 <= a.nL; t += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int o = (t + u) / L.S;
              v[u] = (double)cl.map_shared_rank(reinterpret_cast<T*>(sm + L.o_b), o)[t + u - o * L.S];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) s = fma(iv[(long long)li * a.nL + t + u], v[u], s);
          }
          for (; t < a.nL; ++t) {
            const int o = t / L.S;
            const T* bb = cl.map_shared_rank(reinterpret_cast<T*>(sm + L.o_b), o);
            s = fma(iv[(long long)li * a.nL + t], (double)bb[t - o * L.S], s);
          }
        }
        x[li] = (T)s;
      }
    }
    // (without the direct solve x = omega M^-1 b is already there)
  }
  // up: prolongation x_l += P x_{l+1}, then post-relaxation into r_l
  for (int l = nt - 2; l >= 0; --l) {
    const CTailLevel& L = a.lev[l];
    const CTailLevel& C = a.lev[l + 1];
    const char* ro = sm + a.vec_bytes;
    const int xcoff = (l + 1 == nt - 1) ? C.o_x : C.o_r;  // the corrected x of level l+1
    const unsigned short* pc = reinterpret_cast<const unsigned short*>(ro + L.o_pcol);
    const T* pv = reinterpret_cast<const T*>(ro + L.o_pval);
    T* x = reinterpret_cast<T*>(sm + L.o_x);
    ctail_sync();  // x of level l+1 complete
    for (int li = tid; li < L.S; li += CT) {
      T v = x[li];
      v = fma(pv[li], ctail_get<T>(cl, sm, xcoff, pc[li]), v);
      v = fma(pv[L.S + li], ctail_get<T>(cl, sm, xcoff, pc[L.S + li]), v);
      x[li] = v;
    }
    ctail_sync();  // x + P e of level l complete
    const int* rp = reinterpret_cast<const int*>(ro + L.o_rowptr);
    const unsigned short* col = reinterpret_cast<const unsigned short*>(ro + L.o_col);
    const T* val = reinterpret_cast<const T*>(ro + L.o_val);
    const T* dv = reinterpret_cast<const T*>(ro + L.o_dinv);
    const T* b = reinterpret_cast<const T*>(sm + L.o_b);
    T* out = reinterpret_cast<T*>(sm + L.o_r);
    ctail_apply<T>(cl, sm, L.o_x, L, rp, col, val,
                   [&](int li, T ax) { out[li] = fma(dv[li], b[li] - ax, x[li]); });
  }
  // the corrected x of level T (own slice) to global memory; its rows were
  // written by the first lanes of the row groups
  __syncthreads();
  {
    const CTailLevel& L = a.lev[0];
    const T* res = reinterpret_cast<const T*>(sm + (nt > 1 ? L.o_r : L.o_x));
    for (int li = tid; li < L.S; li += CT) {
      const int g = c * L.S + li;
      if (g < L.n) x_top[g] = res[li];
    }
  }
  ctail_sync();  // no CTA leaves while another may still read its shared memory
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class T>
bool ctail_query(int nc, long long smem);
void launch_ctail_rowlen(const std::vector<Level>& lev, int first, int last, int* const* len,
                         cudaStream_t st) {
  for (int l0 = first; l0 <= last; l0 += SSAMG_CTAIL_MAX_LEVELS) {
    CTailRowlenArgs a{};
    int nb = 0;
    for (int l = l0; l <= last && a.nl < SSAMG_CTAIL_MAX_LEVELS; ++l) {
      a.b0[a.nl] = nb;
      a.len[a.nl] = len[l - first];
      a.lv[a.nl] = lev[l].view<double>();
      ++a.nl;
      nb += cdiv(lev[l].N, 8);
    }
    a.b0[a.nl] = nb;
    if (nb == 0) continue;
    k_ctail_rowlen<<<nb, 256, 0, st>>>(a);
    SSAMG_LAUNCH_CHECK();
  }
}

void launch_ctail_fill(bool fp32, const std::vector<Level>& lev, int t0, const CTailArgs& ta,
                       const double* inv, char* image, long long ro_bytes, cudaStream_t st) {
  const int nt = ta.nt;
  CTailFillArgs a{};
  a.nl = nt;
  a.nL = ta.nL;
  a.ro_bytes = ro_bytes;
  a.image = image;
  int nb = 0;
  for (int j = 0; j < nt; ++j) {
    const Level& L = lev[t0 + j];
    CTailFillLevel& v = a.lev[j];
    v.L = L.view<double>();
    v.fm = j > 0 ? lev[t0 + j - 1].view<double>() : v.L;
    v.ln = j + 1 < nt ? lev[t0 + j + 1].view<double>() : v.L;
    v.has_fm = j > 0;
    v.has_p = j + 1 < nt;
    v.dinv = L.dinv;
    v.inv = (j + 1 == nt) ? inv : nullptr;
    v.lv = ta.lev[j];
    v.Sm = j > 0 ? ta.lev[j - 1].S : 1;
    v.Sn = j + 1 < nt ? ta.lev[j + 1].S : 1;
    a.b0[j] = nb;
    nb += cdiv(L.N, 8);
  }
  a.b0[nt] = nb;
  if (fp32)
    k_ctail_fill<float><<<nb, 256, 0, st>>>(a);
  else
    k_ctail_fill<double><<<nb, 256, 0, st>>>(a);
  SSAMG_LAUNCH_CHECK();
}

template <class T>
bool ctail_prepare(int nc, long long smem) {
  // the answer per device and (nc, smem) is kept: the occupancy query costs
  // more than the rest of a small setup
  static std::mutex mu;
  static std::map<std::tuple<int, int, long long>, bool> known;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const auto key = std::make_tuple(dev, nc, smem);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = known.find(key);
    if (it != known.end()) {
      if (it->second)
        SSAMG_CUDA(cudaFuncSetAttribute(k_ctail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      return it->second;
    }
  }
  const bool ok = ctail_query<T>(nc, smem);
  std::lock_guard<std::mutex> lock(mu);
  known[key] = ok;
  return ok;
}

template <class T>
bool ctail_query(int nc, long long smem) {
  if (cudaFuncSetAttribute(k_ctail<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_ctail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(CT);
  cfg.dynamicSmemBytes = (size_t)smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, k_ctail<T>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return nclusters >= 1;
}

template <class T>
void launch_ctail(const CTailArgs& a, int nc, long long smem, const T* b_top, T* x_top,
                  cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nc);
  cfg.blockDim = dim3(CT);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = g_ssamg_pdl ? 2 : 1;
  SSAMG_CUDA(cudaLaunchKernelEx(&cfg, k_ctail<T>, a, b_top, x_top));
  SSAMG_LAUNCH_CHECK();
}

template bool ctail_prepare<float>(int, long long);
template bool ctail_prepare<double>(int, long long);
template void launch_ctail<float>(const CTailArgs&, int, long long, const float*, float*,
                                  cudaStream_t);
template void launch_ctail<double>(const CTailArgs&, int, long long, const double*, double*,
                                   cudaStream_t);
