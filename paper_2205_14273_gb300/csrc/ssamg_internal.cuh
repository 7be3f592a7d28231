// Internal structures of the SSAMG library (host and device).
//
// Data layout in HBM, per level l:
//   vectors      one contiguous array of N_l values; parts in order, each
//                part's box with i fastest, then j, then k.
//   coefficients one buffer per level; every per-cell (variable) stencil entry
//                of a part is a contiguous array of the part's cells (SoA,
//                entry-major); constant entries are a scalar in the part
//                descriptor.  Levels >= 1 are all variable (Galerkin output).
//   P            two arrays (west / east weight) over the fine points of the
//                coarsened parts only (Section 3.2: coarse points carry 1).
//   U            CSR over the rows that have couplings (row list sorted by
//                cell), plus a dense cell -> row map that only face cells read.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/ssamg.h"

#define SSAMG_MAXE 27
#define SSAMG_BLOCK 256
#define SSAMG_DINV_LEVELS 32  // levels per launch of the smoother-diagonal kernel
#define SSAMG_RHS_GROUP 4  // right-hand sides one thread of the several-right-hand-side cycle kernels takes
#define SSAMG_HOST_THREADS 16  // host threads of the coupling conversion of one call
#define SSAMG_MAX_PART_BOXES 16  // boxes of one part (ssamg_grid_add_box)
#define SSAMG_CPT_LARGE 4         // cells per thread on large levels
#define SSAMG_CPT_MIN_CELLS 300000  // levels smaller than this use one cell per thread
#define SSAMG_TUNE_MARGIN 0.97    // a tuned tile form must save 3% of a level's time
#define SSAMG_TUNE_ITER_MARGIN 0.99  // and the tuned table 1% of a whole PCG iteration
#define SSAMG_EW 4                 // cells per thread of the elementwise pre-relaxation
// Bricks of the checked 7-point operator applies: SSAMG_BRICK_X x _Y threads
// (one column each), marching SSAMG_BRICK_Z cells along z.
#define SSAMG_BRICK_X 32
#define SSAMG_BRICK_Y 8
#define SSAMG_BRICK_Z 8
#define SSAMG_RP_BRICKS 152  // fewest bricks for the restriction / prolongation brick forms
#define SSAMG_RP_FILL 0.8    // and the least fraction of their brick cells inside the parts
#define SSAMG_TPR 4       // fewest lanes per U row in row jobs
#define SSAMG_TPR_MAX 16  // most lanes per U row (levels whose rows are long)

// ---------------------------------------------------------------------------
// Division by a run-time constant (round-up multiply-high method of Granlund
// and Montgomery, PLDI 1994): q = (mulhi(n, m) + n) >> s, exact for every
// n < 2^31 with s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1.
// ---------------------------------------------------------------------------
struct FastDiv {
  unsigned d, m, s;
};

inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  f.d = d ? d : 1;
  unsigned s = 0;
  while ((1ull << s) < f.d) ++s;
  f.s = s;
  f.m = (unsigned)((((1ull << 32) * ((1ull << s) - f.d)) / f.d) + 1ull);
  if (f.d == 1) f.m = 0;
  return f;
}

__host__ __device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
  return (__umulhi(n, f.m) + n) >> f.s;
#else
  return (unsigned)((((unsigned long long)n * f.m >> 32) + n) >> f.s);
#endif
}

// ---------------------------------------------------------------------------
// Per-part, per-level descriptor (device copy).  4-byte multiple, <= 1 KiB so
// one block can stage it in shared memory with a single pass of 256 threads.
// ---------------------------------------------------------------------------
struct DPart {
  long long coef[SSAMG_MAXE];  // element offset of a variable entry, -1: constant
  double cval[SSAMG_MAXE];     // value of a constant entry
  float cval32[SSAMG_MAXE];    // the same rounded to FP32 (converting in the loop would use the FP64 pipe)
  double omega;                // omega_p (Eq. relax1) at this level
  int n[3];                    // extents along x, y, z
  int ncell;
  int off;                     // first cell in the level vector
  int blk0;                    // first block of cell-wise launches over this level
  int nent;
  int dstar;                   // coarsening direction at this level, -1: none
  int par;                     // lo[dstar] & 1 (parity of local cell 0)
  int has_u;                   // 0: no U couplings; 1: rows on the box faces only; 2: rows inside too
  int coff;                    // first cell of the part in the next level vector
  int cn[3];                   // extents on the next level
  int cncell;
  int poff;                    // first fine point in this level's P arrays
  int nf[3];                   // extents of the fine-point grid
  int nfine;
  int fblk0;                   // first block of launches over fine points
  int cpt;                     // cells per thread of this level's tiles (tile = cpt x block)
  int allvar;                  // every entry per cell, entry e at coef[coef[0] + e * ncell + c]
  int canon27;                 // 27 entries in offset-code order (entry e has code e)
  unsigned varmask;            // bit e: entry e is per cell
  int zeroext;                 // per-cell entries are exactly zero where c + o leaves the box
  int prob;                    // problem of the part (a batch of independent problems)
  int skip;                    // relaxation turned off at this level (Section 3.4 "skip")
  int bblk0;                   // first block of brick launches over this level
  int bb[3];                   // bricks along x, y, z (SSAMG_BRICK_X x _Y x _Z cells each)
  FastDiv dx, dxy;             // divide by n[0], n[0]*n[1]
  FastDiv cdx, cdxy;           // same on the next level
  FastDiv fdx, fdxy;           // same on the fine-point grid
  int disp[SSAMG_MAXE];        // linear displacement of each entry
  signed char o[SSAMG_MAXE][3];
  signed char slot[27];        // entry index of offset code (ox+1)+3(oy+1)+9(oz+1), -1 absent
  signed char uent[SSAMG_MAXE];  // level 0: the user's index of entry e (gradient output order)
  signed char pad_[2];
};
static_assert(sizeof(DPart) % 4 == 0 && sizeof(DPart) <= 1024, "DPart layout");

// Scalars of one PCG solve (device memory).
struct PcgScalars {
  double tol, bb, rr, rz, pq, alpha, beta, tol2bb;
  int iter, max_iter, status, flexible, done, pad_;
};
// The PCG scalars while a solve's kernels are enqueued (level views carry
// them, see LevelView::skip), else null (per host thread).
extern thread_local const PcgScalars* g_ssamg_skip;

// Loop control of a (batched) PCG solve: the ticket of the per-problem final
// kernel and whether any problem still iterates.
struct PcgCtl {
  unsigned ticket;
  int active;
};

// Device state the PCG launchers share: one PcgScalars per problem, the
// level-0 block range of each problem (pb[0..nprob], and pbb[0..nprob] for
// brick launches) and the block partials.
struct PcgCtx {
  const int* pb;
  const int* pbb;  // the same in brick blocks (the level-0 brick launches' partials)
  int nprob;
  PcgScalars* sc;
  PcgCtl* ctl;
  double* partial;
  double* hist;    // per problem ||r_k||^2, k = 0..hstride-1 (residual history)
  int hstride;
  // the scalars whose done flags decide whether the solve goes on: sc and
  // nprob, or those of every right-hand side solved together
  const PcgScalars* any_sc;
  int any_n;
};

// Views passed to kernels by value.
template <class T>
struct LevelView {
  const DPart* parts;
  const int* blk;        // np + 1 block starts of cell-wise launches
  const int* bblk;       // np + 1 block starts of brick launches
  const int* fblk;       // np + 1 block starts of fine-point launches
  const int* cellstart;  // np + 1 first cells
  int np;
  int N;
  const T* coef;
  const T* dinv;
  const T* Pw;
  const T* Pe;
  const int* u_map;
  const int* u_ptr;
  const int* u_col;
  const T* u_val;
  const unsigned char* u_bits;
  const int* u_rows;
  const int* u_pj;      // per coupling: the (<= 2) coarse columns of P's row of its column cell
  const T* u_pw;        // and their weights (-1 column: absent)
  const int* u_rj;      // per coupling (levels >= 1): the (<= 3) fine cells of P^T's row of its
  const T* u_rw;        // column cell (centre, -d*, +d*; -1 absent) and the two side weights
  T* uy;                // dense per-cell (U x)(c) of the vector last passed to a row job; 0 off rows
  int nr;
  int nublk;            // blocks of row jobs (SSAMG_BLOCK / tpr rows each)
  int tpr;              // lanes per U row in row jobs (4, 8 or 16)
  // inside a PCG solve: the problems' scalars; a block of a problem whose
  // iteration has stopped leaves its cycle work undone (nothing reads it)
  const PcgScalars* skip;
  // right-hand sides one launch takes together (1 elsewhere): block b works
  // on tile b / nrhs for right-hand side j = b % nrhs, whose vectors and U x
  // lie vstride elements after those of j - 1 and whose scalars skip_stride
  // entries after them
  int nrhs;
  int skip_stride;
  long long vstride;
};

// One level of the fused coarse tail: the level's view and its cycle vectors.
#define SSAMG_TAIL_MAX_CELLS 32768  // levels at most this large run in the fused tail
#define SSAMG_TAIL_MAX_PARTS 8
#define SSAMG_TAIL_BLOCK 256
#define SSAMG_TAIL_MAX_BLOCKS 128
#define SSAMG_TAIL_CTA 1024         // threads of the single-CTA tail
#define SSAMG_TAIL_CTA_CELLS 4096   // default largest level of the single-CTA tail
#define SSAMG_BARRIER_SPINS (1u << 24)  // default poll cap: ~1 s of polling before a barrier gives up

// Coarse-level transition run by one thread-block cluster (kernels_tail.cu):
// per tail level, the rows are split into slices of S rows, one per CTA; a
// column index packs the owning CTA (high bits) and the position in its slice
// (SSAMG_CTAIL_LOCAL_BITS low bits).  Offsets are in bytes: vectors within the
// CTA's vector region, the rest within its read-only region (its image).
#define SSAMG_CTAIL_THREADS 512
#define SSAMG_CTAIL_MAX_LEVELS 32
#define SSAMG_CTAIL_LOCAL_BITS 12
#define SSAMG_CTAIL_MAX_CTAS 16
#define SSAMG_CTAIL_CELLS 4096  // default largest level of the cluster tail
struct CTailLevel {
  int n, S;                  // cells, rows per CTA slice
  int tpr;                   // lanes per CSR row in the operator applies (power of two <= 32)
  int o_x, o_b, o_r;         // the level's vectors
  int o_rowptr, o_col, o_val, o_dinv;  // CSR of A = S + U (local row pointers), omega M^-1
  int o_pcol, o_pval;        // P's row of each fine cell (2 per row), to the next level
  int o_rcol, o_rval;        // restriction row of each coarse cell (3 per row), from the level above
  int o_inv;                 // coarsest level: rows of the explicit inverse (FP64)
};
struct CTailArgs {
  const char* image;         // NC images of ro_bytes each
  long long ro_bytes;
  int vec_bytes;
  int nt;                    // tail levels (>= 2)
  int direct;                // 1: coarsest level by the explicit inverse, 0: one relaxation sweep
  int nL;                    // cells of the coarsest level
  CTailLevel lev[SSAMG_CTAIL_MAX_LEVELS];
};

// Grid barrier state (device memory): the arrival counter, the poll cap
// after which a waiting block gives up, the sticky failure flag, and arrivals
// expected beyond the launch's own blocks (0; a self-test sets more, so that
// the wait cannot complete and must end at the cap).
struct TailBarrier {
  unsigned count;
  unsigned cap;
  int err;
  int extra;
};
template <class T>
struct TailLevel {
  LevelView<T> L;
  T* x;
  T* b;
  T* r;
  T* t;
  int shape;  // StencilShape of the level's operator apply
  int pad_;
};

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct PartH {
  int lo[3], hi[3], n[3];
  long long ncell;
  int off;
  int dstar, par;
  double omega;
  int nent;
  int o[SSAMG_MAXE][3];
  int var[SSAMG_MAXE];
  double cval[SSAMG_MAXE];
  long long coef_off[SSAMG_MAXE];
  int uent[SSAMG_MAXE];  // level 0: the user's entry index of entry e (coarse levels: e)
  int nf[3];
  long long nfine;
  int poff;
  int has_u;
  int skip;  // relaxation turned off on this part at this level (Section 3.4 "skip")
};

struct Arena {
  std::vector<std::pair<char*, size_t>> chunks;
  size_t cur = 0, used = 0;
  void reset() { cur = 0; used = 0; }
  void* alloc(size_t bytes);  // 256-byte aligned, throws on failure
  void release();
  ~Arena() { release(); }
};

struct Level {
  int np = 0;
  long long guard = 0;  // zeroed cells before and after every internal level vector
  long long N = 0;
  std::vector<PartH> parts;
  std::vector<DPart> dparts;
  DPart* d_parts = nullptr;
  int* d_blk = nullptr;
  int* d_bblk = nullptr;
  int* d_fblk = nullptr;
  int* d_cellstart = nullptr;
  int nblk = 0, nfblk = 0, nbblk = 0;
  int cpt = 1;
  int bricks = 1; // 0: the tile table keeps this level's operator applies on cell tiles
  double brick_fill = 0.0;  // cells / (bricks x brick cells): how full the level's bricks are
  int kvar = 2;   // per-cell stencil entries: 0 none, 1 only diagonals, 2 others too
  int shape = 0;  // StencilShape of the level's operator apply
  std::vector<int> hblk;  // host copy of the block starts of cell-wise launches
  std::vector<int> hbblk; // and of brick launches
  double* coef = nullptr;
  float* coef32 = nullptr;
  long long ncoef = 0;
  double* Pw = nullptr;
  double* Pe = nullptr;
  float* Pw32 = nullptr;
  float* Pe32 = nullptr;
  long long nP = 0;
  double* dinv = nullptr;
  float* dinv32 = nullptr;
  int nr = 0;
  long long nnz = 0;
  int* u_ptr = nullptr;
  int* u_rows = nullptr;
  int* u_col = nullptr;
  int* u_map = nullptr;
  double* u_val = nullptr;
  float* u_val32 = nullptr;
  unsigned char* u_bits = nullptr;
  int* u_pj = nullptr;
  double* u_pw = nullptr;
  float* u_pw32 = nullptr;
  int* u_rj = nullptr;
  double* u_rw = nullptr;
  float* u_rw32 = nullptr;
  double* uy64 = nullptr;
  float* uy32 = nullptr;
  int nublk = 0;
  int tpr = SSAMG_TPR;
  // cycle work vectors (precision of the cycle)
  void* x = nullptr;
  void* b = nullptr;
  void* r = nullptr;
  void* t = nullptr;

  template <class T>
  LevelView<T> view() const;
};

template <>
inline LevelView<double> Level::view<double>() const {
  return LevelView<double>{d_parts, d_blk, d_bblk, d_fblk, d_cellstart, np, (int)N, coef, dinv, Pw, Pe,
                           u_map, u_ptr, u_col, u_val, u_bits, u_rows, u_pj, u_pw, u_rj, u_rw, uy64, nr,
                           nublk, tpr, g_ssamg_skip, 1, 0, 0};
}
template <>
inline LevelView<float> Level::view<float>() const {
  return LevelView<float>{d_parts, d_blk, d_bblk, d_fblk, d_cellstart, np, (int)N, coef32, dinv32, Pw32,
                          Pe32, u_map, u_ptr, u_col, u_val32, u_bits, u_rows, u_pj, u_pw32, u_rj,
                          u_rw32, uy32, nr, nublk, tpr, g_ssamg_skip, 1, 0, 0};
}

struct SsamgError {
  int code;
  std::string msg;
};

#define SSAMG_CUDA(call)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) throw SsamgError{SSAMG_ERR_CUDA, std::string(#call ": ") +       \
                                                           cudaGetErrorString(e_)};         \
  } while (0)

// Every kernel launch of the library passes through this check, which also
// counts it (per host thread) for the launch statistics.
extern thread_local long long g_ssamg_launches;
// Nonzero while an entry point enqueues solve kernels with programmatic
// dependent launch (per host thread; set by the entry point, read by the
// launchers).
extern thread_local int g_ssamg_pdl;
// Nonzero while the entry point allows brick launches for checked 7-point
// levels (per host thread, like g_ssamg_pdl).
extern thread_local int g_ssamg_bricks;

#define SSAMG_LAUNCH_CHECK()       \
  do {                             \
    ++g_ssamg_launches;            \
    SSAMG_CUDA(cudaGetLastError()); \
  } while (0)

// ---------------------------------------------------------------------------
// Kernel launchers (kernels_*.cu)
// ---------------------------------------------------------------------------
// setup
void launch_wsum(const Level& L, double* partial, double* c_out, cudaStream_t st);
// Device address of the static block-partial scratch of the allocation-free
// coupling sums (SSAMG_NOALLOC_MAX_BLOCKS x 3 doubles) on the current device.
double* wsum_static_scratch();
void launch_interp(const Level& F, bool fp32, cudaStream_t st);
void launch_rap_struct(const Level& F, const Level& Cl, bool fp32, cudaStream_t st);
// P^T U P (Section 3.3): P rows of the fine coupling rows (prI, prW, prA: two
// per row) and the marker of the coarse rows; the coarse rows' fine-row table
// (fr, frw: three per coarse row); the per-row entry counts and the fill.
// F.u_pj / F.u_pw (P rows of the coupling columns) must be computed first.
void launch_uprow(const Level& F, const Level& Cl, int* prI, double* prW, signed char* prA,
                  int* marker, cudaStream_t st);
void launch_urows(const Level& Cl, const int* scan, const int* marker, cudaStream_t st);
void launch_frows(const Level& F, const Level& Cl, const int* prI, const double* prW,
                  const signed char* prA, int* fr, double* frw, cudaStream_t st);
// lists: 2 (Cl.nr + 1) ints (the rows the counting pass lists for the warp
// forms of the merge, reused by the fill pass).
// Staging of the rows of U_c = P^T U P (sorted once, copied once counted).
struct UStage {
  int* toff;    // first staging slot of each coarse row
  int* cursor;  // next free staging slot
  int* col;
  double* val;
  unsigned char* bits;
};
void launch_usort(const Level& F, const Level& Cl, int* lists, const int* fr,
                  const double* frw, int* counts, const UStage& t, int* err, cudaStream_t st);
void launch_ucopy(const Level& F, const Level& Cl, const UStage& t, bool fp32, cudaStream_t st);
// Smoother diagonals of levels first..last in one launch (per SSAMG_DINV_LEVELS).
void launch_dinv(const std::vector<Level>& lev, int first, int last, int relax, double factor,
                 bool fp32, cudaStream_t st);
void launch_to_float(const double* in, float* out, long long n, cudaStream_t st);
// zero the values of a per-cell entry with offset o where c + o leaves the box
void launch_mask_outside(double* vals, const int n[3], const int o[3], cudaStream_t st);
// The boxes of a part of several boxes, relative to its bounding box's
// corner: b[t] = (lo x, y, z, hi x, y, z).
struct PartBoxes {
  int n;
  int b[SSAMG_MAX_PART_BOXES][6];
};
// Entry with offset o of a part held over its bounding box (extents n):
// the diagonal (o = 0) becomes 1 at cells outside the boxes, any other entry
// 0 where the cell or its neighbour c + o is outside them.
void launch_mask_part(double* vals, const int n[3], const int o[3], const PartBoxes& pb,
                      cudaStream_t st);
void launch_coarse_assemble(const Level& L, double* A, cudaStream_t st);
void launch_cholesky(int n, double* A, int* status, cudaStream_t st);
// exclusive scan of n ints in place; returns nothing (total at out[n])
void launch_scan(int* data, long long n, int* tmp, cudaStream_t st);
// Device memory pool (abi.cu): blocks are cached per rounded size; free a
// block only after pool_fence() once no kernel can still use it.
void* pool_alloc(size_t bytes);
void pool_free(void* p);
void pool_fence();
// Level-0 coupling CSR (kernels_setup.cu): m tuples in, rows ascending,
// columns ascending per row, duplicates summed in input order; the outputs
// hold at least m entries (N + 1 for u_map's N).  Synchronises st.
struct UAssemble {
  int N;
  long long m;
  const int* row;
  const int* col;
  const double* val;
  const unsigned char* bits;
  int* u_rows;
  int* u_ptr;
  int* u_col;
  double* u_val;
  unsigned char* u_bits;
  int* u_map;
};
void launch_uassemble(const UAssemble& a, int* nr, long long* nnz, cudaStream_t st);
size_t scan_tmp_ints(long long n);

// cycle (T = float or double)
template <class T>
void launch_relax0(const Level& L, const T* b, T* x, cudaStream_t st);
// x = omega M^-1 b and, in the same launch, uy = U x (row jobs)
template <class T>
void launch_relax0_u(const Level& L, const T* b, T* x, cudaStream_t st);
// xout = xin + P ec and uy = U xout (row jobs)
template <class T>
void launch_prolong_u(const Level& F, const T* ec, const T* xin, T* xout, cudaStream_t st);
// uy = U x
template <class T>
void launch_uy(const Level& L, const T* x, cudaStream_t st);
// first pre-relaxation from the FP64 residual (b0 = (T) r) and last
// post-relaxation into the FP64 z with the PCG's r.z partials (2 per block)
template <class T>
void launch_relax0_u_first(const Level& L, const double* r64, T* b0, T* x, cudaStream_t st);
template <class T>
void launch_relax_final(const Level& L, const T* x, const T* b, double* z, const double* rpcg,
                        double* zprev, double* partial, cudaStream_t st);
// row-job setup data of L's couplings: P rows (L.u_pj set) and restriction
// rows from the level above Fp (L.u_rj set)
void launch_ucols(const Level* Fp, const Level& L, bool fp32, bool pj, bool rj, cudaStream_t st);
template <class T>
void launch_residual(const Level& L, const T* x, const T* b, T* r, cudaStream_t st);
template <class T>
void launch_relax(const Level& L, const T* x, const T* b, T* xo, cudaStream_t st);
// the same for R right-hand sides in one launch (cell-tile levels only)
template <class T>
void launch_residual_rhs(const Level& L, int R, long long vstride, int skip_stride, const T* x,
                         const T* b, T* r, cudaStream_t st);
template <class T>
void launch_relax_rhs(const Level& L, int R, long long vstride, int skip_stride, const T* x,
                      const T* b, T* xo, cudaStream_t st);
template <class T>
void launch_restrict(const Level& F, const Level& Cl, const T* r, T* bc, T* xc, cudaStream_t st);
template <class T>
void launch_prolong(const Level& F, const Level& Cl, const T* ec, T* x, cudaStream_t st);
template <class T>
void launch_coarse_solve(int n, const double* Lfac, const T* b, T* x, cudaStream_t st);
// Levels lt..Lc of the V-cycle in one single-block launch (down sweep from
// b of level lt, coarsest solve, up sweep; result in t of level lt).
template <class T>
void launch_vtail(const TailLevel<T>* lv, int nlev, const double* cinv, int nL, int coarse_direct,
                  int nblocks, TailBarrier* gb, cudaStream_t st, int nparts);
// Allows the single-CTA tail its shared memory (level table + part
// descriptors); false when they do not fit.
template <class T>
bool vtail_one_prepare(int nlev, int nparts);
int tail_max_blocks();
// Self-test of the bounded grid barrier: nblocks co-resident blocks meet at
// one barrier that also waits for `extra` arrivals that never come (when
// extra > 0), polling at most `cap` times.  Returns the barrier's failure
// flag (1: a block gave up).  Synchronises st.
int barrier_selftest(int nblocks, int extra, unsigned cap, cudaStream_t st);
void launch_coarse_inverse(int n, const double* Lfac, double* inv, cudaStream_t st);
// cluster tail (kernels_tail.cu)
// Row lengths of levels first..last (len[l - first]: N_l ints each) and the
// images of the tail levels t0 .. t0 + ta.nt - 1, each in one launch.
void launch_ctail_rowlen(const std::vector<Level>& lev, int first, int last, int* const* len,
                         cudaStream_t st);
void launch_ctail_fill(bool fp32, const std::vector<Level>& lev, int t0, const CTailArgs& ta,
                       const double* inv, char* image, long long ro_bytes, cudaStream_t st);
// Allows the tail kernel nc-CTA clusters and smem bytes of shared memory per
// CTA; false when the device cannot run such a cluster.
template <class T>
bool ctail_prepare(int nc, long long smem);
template <class T>
void launch_ctail(const CTailArgs& a, int nc, long long smem, const T* b_top, T* x_top,
                  cudaStream_t st);
template <class T>
void launch_coarse_apply(int n, const double* inv, const T* b, T* x, cudaStream_t st);
void launch_cast_d2f(const double* in, float* out, long long n, cudaStream_t st);
void launch_cast_f2d(const float* in, double* out, long long n, cudaStream_t st);
void launch_fill(double* x, long long n, double v, cudaStream_t st);
// y = A_l x; x may be a caller vector without guard cells
void launch_matvec(const Level& L, const double* x, double* y, cudaStream_t st);

// PCG (FP64)
void launch_pcg_init(const Level& L, const double* b, const double* x, double* r,
                     const PcgCtx& c, cudaStream_t st);
void launch_pcg_start(const Level& L0, const double* r, const double* z, double* p, double* zprev,
                      const PcgCtx& c, cudaStream_t st);
void launch_pcg_beta(const Level& L0, const double* r, const double* z, double* zprev, double* p,
                     const PcgCtx& c, cudaStream_t st);
void launch_pcg_beta_from_partials(const Level& L0, const double* z, double* p, const PcgCtx& c,
                                   const int* ranges, cudaStream_t st);
// Whether L's operator applies run over bricks, and the per-problem ranges of
// the partials those launches write.
bool uses_bricks(const Level& L);
bool rp_bricks(const Level& L);
const int* partial_ranges(const Level& L, const PcgCtx& c);
// block ranges of the dot partials the cycle's last relaxation writes
const int* final_ranges(const Level& L, const PcgCtx& c);
void launch_pcg_alpha(const Level& L, const double* p, double* q, const PcgCtx& c,
                      cudaStream_t st);
void launch_pcg_update(const Level& L0, const double* p, const double* q, double* x, double* r,
                       const PcgCtx& c, cudaGraphConditionalHandle h, int use_handle,
                       cudaStream_t st);
void launch_true_residual(const Level& L, const double* b, const double* x, double* r,
                          const PcgCtx& c, double* out, cudaStream_t st);

// differentiation
void launch_coef_gradient(const Level& L, const double* lam, const double* x, double* dcoef,
                          cudaStream_t st);
void launch_diffusion_exp_gradient(const Level& L, const double* g, const double* lam,
                                   const double* x, double* dg, double* kap, cudaStream_t st);
