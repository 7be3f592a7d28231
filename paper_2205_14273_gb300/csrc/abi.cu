// C ABI of the SSAMG library: grid / matrix / solver objects, the setup
// driver (Sections 3.1-3.4) and the PCG + V(1,1) solve driver (Section 4).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <thread>
#include <unordered_map>

#include <nvtx3/nvToolsExt.h>

#include "ssamg_internal.cuh"

// NVTX range around a scope (entry points, set-up stages and levels): seen by
// profilers that record NVTX, a few nanoseconds otherwise.
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  NvtxRange(const char* prefix, int k) {
    char buf[64];
    std::snprintf(buf, sizeof buf, "%s %d", prefix, k);
    nvtxRangePushA(buf);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

// ---------------------------------------------------------------------------
// Device memory pool: blocks freed by matrices and solvers are kept per
// rounded size and handed to the next allocation of that size, so objects
// created and destroyed per step (a new matrix and solver every time) do not
// pay cudaMalloc / cudaFree each time.  Sizes round up to a power of two
// below 1 MiB and to 2 MiB multiples above.  Callers free only after
// pool_fence() (a device synchronisation, which cudaFree would have done),
// so a block is never handed out while a kernel may still use it.  On an
// allocation failure the cache is released and the allocation retried;
// ssamg_release_device_cache() returns the cache to the driver.
// ---------------------------------------------------------------------------
namespace {
struct DevPool {
  std::mutex m;
  std::multimap<size_t, void*> cache;   // rounded size -> free block
  std::unordered_map<void*, size_t> live;
  size_t cached = 0;
};
DevPool& dev_pool() {
  static DevPool* p = new DevPool;  // outlives every object (no order-of-destruction issue)
  return *p;
}
size_t pool_round(size_t b) {
  if (b <= (size_t(1) << 20)) {
    size_t r = 512;
    while (r < b) r <<= 1;
    return r;
  }
  const size_t g = size_t(2) << 20;
  return (b + g - 1) / g * g;
}
void pool_trim(DevPool& P) {
  for (auto& kv : P.cache) cudaFree(kv.second);
  P.cache.clear();
  P.cached = 0;
}
}  // namespace

void* pool_alloc(size_t bytes) {
  DevPool& P = dev_pool();
  const size_t r = pool_round(std::max<size_t>(bytes, 1));
  std::lock_guard<std::mutex> lk(P.m);
  auto it = P.cache.find(r);
  if (it != P.cache.end()) {
    void* q = it->second;
    P.cache.erase(it);
    P.cached -= r;
    P.live[q] = r;
    return q;
  }
  void* q = nullptr;
  if (cudaMalloc(&q, r) != cudaSuccess) {
    cudaGetLastError();
    cudaDeviceSynchronize();
    pool_trim(P);
    if (cudaMalloc(&q, r) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  }
  P.live[q] = r;
  return q;
}

void pool_fence() { cudaDeviceSynchronize(); }

void pool_free(void* q) {
  if (!q) return;
  DevPool& P = dev_pool();
  std::lock_guard<std::mutex> lk(P.m);
  auto it = P.live.find(q);
  if (it == P.live.end()) return;
  P.cache.emplace(it->second, q);
  P.cached += it->second;
  P.live.erase(it);
}


// Pinned host buffers of destroyed solvers are kept the same way (per
// rounded size): cudaMallocHost costs far more than a small set-up step.
namespace {
struct HostPool {
  std::mutex m;
  std::multimap<size_t, void*> cache;
  std::unordered_map<void*, size_t> live;
};
HostPool& host_pool() {
  static HostPool* p = new HostPool;
  return *p;
}
}  // namespace

void* pinned_alloc(size_t bytes) {
  HostPool& P = host_pool();
  const size_t r = pool_round(std::max<size_t>(bytes, 1));
  std::lock_guard<std::mutex> lk(P.m);
  auto it = P.cache.find(r);
  void* q = nullptr;
  if (it != P.cache.end()) {
    q = it->second;
    P.cache.erase(it);
  } else if (cudaMallocHost(&q, r) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  P.live[q] = r;
  return q;
}

// Only after the work that reads or writes the buffer has finished.
void pinned_free(void* q) {
  if (!q) return;
  HostPool& P = host_pool();
  std::lock_guard<std::mutex> lk(P.m);
  auto it = P.live.find(q);
  if (it == P.live.end()) return;
  P.cache.emplace(it->second, q);
  P.live.erase(it);
}

template <class T>
T* pinned_new(long long n) {
  T* q = (T*)pinned_alloc(sizeof(T) * (size_t)std::max<long long>(n, 1));
  if (!q) throw SsamgError{SSAMG_ERR_OOM, "pinned host allocation failed"};
  return q;
}

extern "C" long long ssamg_release_device_cache(void) {
  DevPool& P = dev_pool();
  std::lock_guard<std::mutex> lk(P.m);
  const long long n = (long long)P.cached;
  pool_trim(P);
  HostPool& H = host_pool();
  std::lock_guard<std::mutex> lh(H.m);
  for (auto& kv : H.cache) cudaFreeHost(kv.second);
  H.cache.clear();
  return n;
}

template <class T>
T* pool_new(long long n) {
  T* q = (T*)pool_alloc(sizeof(T) * (size_t)std::max<long long>(n, 1));
  if (!q) throw SsamgError{SSAMG_ERR_OOM, "device allocation failed"};
  return q;
}

// ---------------------------------------------------------------------------
// Arena: chunked bump allocator.  A setup with the same sizes as the previous
// one walks the same chunks in the same order and allocates nothing.
// ---------------------------------------------------------------------------
void* Arena::alloc(size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  while (cur < chunks.size()) {
    if (used + bytes <= chunks[cur].second) {
      void* p = chunks[cur].first + used;
      used += bytes;
      return p;
    }
    ++cur;
    used = 0;
  }
  size_t sz = std::max(bytes, size_t(64) << 20);
  char* p = (char*)pool_alloc(sz);
  if (!p) throw SsamgError{SSAMG_ERR_OOM, "device allocation failed"};
  chunks.push_back({p, sz});
  cur = chunks.size() - 1;
  used = bytes;
  return p;
}

void Arena::release() {
  if (!chunks.empty()) pool_fence();
  for (auto& c : chunks) pool_free(c.first);
  chunks.clear();
  cur = used = 0;
}

// ---------------------------------------------------------------------------
// Objects
// ---------------------------------------------------------------------------
struct ssamg_grid_s {
  int ndim = 3, nparts = 0;
  std::vector<std::array<int, 3>> lo, hi;  // each part's (bounding) box
  std::vector<char> set;
  // a part of several boxes (Section 2): its boxes (lo, hi), empty for a
  // one-box part; the part is held over their bounding box lo..hi
  std::vector<std::vector<std::array<int, 6>>> boxes;
  bool in_part(int p, const int* c) const {
    if (boxes[p].empty()) return true;
    for (const auto& b : boxes[p])
      if (c[0] >= b[0] && c[0] <= b[3] && c[1] >= b[1] && c[1] <= b[4] && c[2] >= b[2] &&
          c[2] <= b[5])
        return true;
    return false;
  }
  bool in_box(int p, const int* c) const {
    for (int d = 0; d < 3; ++d)
      if (c[d] < lo[p][d] || c[d] > hi[p][d]) return false;
    return true;
  }
  bool assembled = false;
  std::vector<long long> off;  // nparts + 1
  long long N = 0;
  long long ncell(int p) const {
    long long n = 1;
    for (int d = 0; d < 3; ++d) n *= hi[p][d] - lo[p][d] + 1;
    return n;
  }
};

struct ssamg_matrix_s {
  ssamg_grid g = nullptr;
  int nent = 0;
  int o[SSAMG_MAXE][3];
  std::vector<std::vector<double>> cval;      // [part][entry]
  std::vector<std::vector<double*>> tmpvar;   // device values set but not yet packed
  std::vector<std::vector<char>> isset, isvar;
  // couplings (host, appended)
  // couplings as added: global row and column cell, direction bits (bit 2d:
  // +d, 2d+1: -d), value; and per part 1 / 2 once a row lies on a face /
  // inside the box
  std::vector<int> c_row, c_col;
  std::vector<unsigned char> c_bits;
  std::vector<double> c_val;
  std::vector<char> c_hasu;
  // assembled (device)
  bool assembled = false;
  double* coef = nullptr;
  long long ncoef = 0;
  std::vector<std::vector<long long>> coef_off;  // [part][entry], -1 const
  int nr = 0;
  long long nnz = 0;
  int *u_rows = nullptr, *u_ptr = nullptr, *u_col = nullptr, *u_map = nullptr;
  double* u_val = nullptr;
  unsigned char* u_bits = nullptr;
  std::vector<char> has_u;
  int version = 0;
  void free_device() {
    if (coef || u_rows) pool_fence();
    pool_free(coef);
    pool_free(u_rows);
    pool_free(u_ptr);
    pool_free(u_col);
    pool_free(u_map);
    pool_free(u_val);
    pool_free(u_bits);
    coef = nullptr;
    u_rows = u_ptr = u_col = u_map = nullptr;
    u_val = nullptr;
    u_bits = nullptr;
  }
  ~ssamg_matrix_s() {
    pool_fence();
    free_device();
    for (auto& v : tmpvar)
      for (auto* p : v) pool_free(p);
  }
};

struct GraphSet {
  cudaGraphExec_t pcg = nullptr;
  cudaGraphExec_t vcycle = nullptr;
  cudaGraphExec_t rounds = nullptr;  // several right-hand sides in one graph
  const double* rounds_b = nullptr;   // the user vectors baked into `rounds`
  double* rounds_x = nullptr;
  int rounds_n = 0;
  int rounds_zero = 1;                // 1: x0 = 0 baked in, 0: x0 read from x
  void reset() {
    if (pcg) cudaGraphExecDestroy(pcg);
    if (vcycle) cudaGraphExecDestroy(vcycle);
    if (rounds) cudaGraphExecDestroy(rounds);
    pcg = vcycle = rounds = nullptr;
    rounds_b = nullptr;
    rounds_x = nullptr;
    rounds_n = 0;
  }
};

// Copies of the per-solve vectors for right-hand sides solved together: on
// every level whose cycle vectors the per-level kernels use, and for the
// FP64 PCG, R slices of each vector (guard cells around each slice), the
// slices of one vector `stride` elements apart; per right-hand side a
// block-partial buffer, the problems' scalars (contiguous: right-hand side
// j's at sc + j nprob) and a residual history.
struct RhsSet {
  int R = 0;                          // right-hand sides of the current solve
  int cap = 0;                        // slices allocated (>= R)
  int nlev = 0;                       // levels 0..nlev-1 carry slices
  std::vector<long long> stride;      // per level, elements between slices
  std::vector<char*> x, b, r, t;      // per level: the first slice
  std::vector<float*> uy32;           // per level: the first U x slice (or none)
  std::vector<double*> uy64;
  long long stride0 = 0;              // the FP64 PCG vectors
  double *pb = nullptr, *px = nullptr, *pr = nullptr, *pz = nullptr, *pp = nullptr,
         *pq = nullptr, *pzprev = nullptr;
  double* partial = nullptr;
  long long partial_len = 0;
  PcgScalars* sc = nullptr;
  double* hist = nullptr;
  long long hist_len = 0;
};

struct ssamg_solver_s {
  ssamg_params prm;
  Arena arena;
  std::vector<Level> lev;
  ssamg_matrix A = nullptr;
  bool ready = false;
  int ndim = 3;
  std::vector<double> c, W;  // nparts x 3
  // coarsest
  int nL = 0;
  double* chol = nullptr;
  double* cinv = nullptr;      // explicit inverse of the coarsest operator (for the fused tail)
  int tail_lt = -1;            // first level of the fused coarse tail (-1: none)
  void* tail_dev = nullptr;    // TailLevel<T> array for levels tail_lt..Lc
  int tail_blocks = 0;
  int tail_parts = 0;          // part descriptors of the tail levels (single-CTA tail)
  TailBarrier* tail_bar = nullptr;
  // cluster tail (use_tail = 3): levels ctail.lev[0..nt) from level ctail_lt on
  int ctail_lt = -1;
  int ctail_nc = 0;
  long long ctail_smem = 0;
  CTailArgs ctail{};
  const TailBarrier tail_bar_init{0u, SSAMG_BARRIER_SPINS, 0, 0};  // host source of its set-up copy
  // PCG work (FP64, level 0 size)
  double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr,
         *zprev = nullptr, *partial = nullptr, *tres = nullptr;
  PcgScalars* sc = nullptr;
  PcgScalars* h_sc = nullptr;  // pinned
  int* h_int = nullptr;        // pinned scratch
  double* h_dbl = nullptr;
  char* h_up = nullptr;        // pinned staging of the level tables (one copy per set-up)
  size_t h_up_cap = 0;
  int* d_err = nullptr;
  // problems: one, or a batch of independent problems in one hierarchy
  int nprob = 1;
  std::vector<int> part_prob;  // problem of each part (empty: all 0)
  std::vector<long long> prob_cells;  // nprob + 1 first cells of each problem
  int* pb = nullptr;           // nprob + 1 level-0 block starts of each problem (device)
  int* pbb = nullptr;          // the same in brick blocks
  PcgCtl* ctl = nullptr;
  double* hist = nullptr;      // residual history: nprob x (max_iter + 1) squared norms
  PcgScalars* sc_init = nullptr;  // nprob starting scalars (tolerance, caps)
  PcgScalars* sc_hist = nullptr;  // per right-hand side copies of sc (multi-round solves)
  double* tres_hist = nullptr;    // and of the true residual sums
  int hist_cap = 0;               // right-hand sides the history holds
  int h_cap = 0;               // problems the pinned buffers hold
  cudaStream_t cs = nullptr;  // capture stream
  cudaStream_t ss = nullptr;  // setup side stream (structured Galerkin products)
  cudaEvent_t ev_p = nullptr, ev_rap = nullptr, ev_rows = nullptr, ev_mark = nullptr,
              ev_uc = nullptr;
  int tiles[SSAMG_TILE_CLASSES] = {};  // tile table by level size class (0: built-in rule)
  std::vector<double> user_W;  // user spacings (3 per part), empty: from the coupling sums
  GraphSet graphs;
  RhsSet rhs;
  // scalars whose done flags decide the solve loop (null: sc, nprob)
  const PcgScalars* any_sc = nullptr;
  int any_n = 0;
  long long setup_launches = 0, head_launches = 0, body_launches = 0;
  ~ssamg_solver_s() {
    graphs.reset();
    if (sc_hist) cudaFree(sc_hist);
    if (tres_hist) cudaFree(tres_hist);
    if (cs) cudaStreamDestroy(cs);
    if (ss) cudaStreamDestroy(ss);
    if (ev_p) cudaEventDestroy(ev_p);
    if (ev_rap) cudaEventDestroy(ev_rap);
    if (ev_rows) cudaEventDestroy(ev_rows);
    if (ev_mark) cudaEventDestroy(ev_mark);
    if (ev_uc) cudaEventDestroy(ev_uc);
    if (h_sc || h_int || h_dbl || h_up) pool_fence();
    pinned_free(h_sc);
    pinned_free(h_int);
    pinned_free(h_dbl);
    pinned_free(h_up);
  }
};

thread_local long long g_ssamg_launches = 0;
thread_local int g_ssamg_pdl = 0;
thread_local int g_ssamg_bricks = 1;
thread_local const PcgScalars* g_ssamg_skip = nullptr;

// While PCG kernels are enqueued: level views carry the problems' scalars,
// so that the cycle kernels of a stopped problem return at once.
struct SkipScope {
  const PcgScalars* old;
  explicit SkipScope(const PcgScalars* sc) : old(g_ssamg_skip) { g_ssamg_skip = sc; }
  ~SkipScope() { g_ssamg_skip = old; }
};

// Enables programmatic dependent launch for the solve kernels an entry point
// enqueues (when the solver's parameters ask for it), and restores the
// previous setting on exit.
struct PdlScope {
  int old, old_b;
  explicit PdlScope(const ssamg_params& prm)
      : old(g_ssamg_pdl), old_b(g_ssamg_bricks) {
    g_ssamg_pdl = prm.use_pdl;
    g_ssamg_bricks = prm.use_bricks;
  }
  ~PdlScope() {
    g_ssamg_pdl = old;
    g_ssamg_bricks = old_b;
  }
};

// Address of the static coupling-sum scratch per device, resolved by setup
// (outside any stream capture) so that the allocation-free entry makes no
// capture-illegal runtime call.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_scratch[kMaxDevices] = {};

double* noalloc_scratch() {
  int dev = 0;
  SSAMG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw SsamgError{SSAMG_ERR_UNSUPPORTED, "device index above 63"};
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_scratch[dev]) g_noalloc_scratch[dev] = wsum_static_scratch();
  return g_noalloc_scratch[dev];
}

namespace {

thread_local std::string g_last_error;

int fail(const SsamgError& e) {
  g_last_error = e.msg;
  return e.code;
}

#define API_BEGIN try {
#define API_END                                       \
  }                                                   \
  catch (const SsamgError& e) { return fail(e); }     \
  catch (const std::bad_alloc&) { return SSAMG_ERR_OOM; }

inline void argcheck(bool ok, const char* msg) {
  if (!ok) throw SsamgError{SSAMG_ERR_ARG, msg};
}

inline long long cdivll(long long a, long long b) { return (a + b - 1) / b; }
inline int floordiv2(int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }
inline int ceildiv2(int v) { return -floordiv2(-v); }

template <class T>
T* aalloc(Arena& a, long long n) {
  return reinterpret_cast<T*>(a.alloc(sizeof(T) * (size_t)std::max<long long>(n, 1)));
}

}  // namespace

// ---------------------------------------------------------------------------
// Status strings
// ---------------------------------------------------------------------------
extern "C" const char* ssamg_status_string(int s) {
  switch (s) {
    case SSAMG_OK: return "ok";
    case SSAMG_NOT_CONVERGED: return "not converged within max_iter";
    case SSAMG_ERR_ARG: return "invalid argument";
    case SSAMG_ERR_STATE: return "call out of order";
    case SSAMG_ERR_OOM: return "out of memory";
    case SSAMG_ERR_CUDA: return "CUDA error";
    case SSAMG_ERR_BREAKDOWN: return "breakdown (non-SPD operator or NaN)";
    case SSAMG_ERR_TIMEOUT: return "device wait timed out";
    case SSAMG_ERR_UNSUPPORTED: return "size limit of this implementation exceeded";
    default: return "unknown status";
  }
}

extern "C" const char* ssamg_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// Grid
// ---------------------------------------------------------------------------
extern "C" int ssamg_grid_create(int ndim, int nparts, ssamg_grid* out) {
  if (!out || ndim < 1 || ndim > 3 || nparts < 1) return SSAMG_ERR_ARG;
  auto* g = new (std::nothrow) ssamg_grid_s;
  if (!g) return SSAMG_ERR_OOM;
  g->ndim = ndim;
  g->nparts = nparts;
  g->lo.assign(nparts, {0, 0, 0});
  g->hi.assign(nparts, {0, 0, 0});
  g->set.assign(nparts, 0);
  g->boxes.assign(nparts, {});
  *out = g;
  return SSAMG_OK;
}

extern "C" int ssamg_grid_set_box(ssamg_grid g, int part, const int lo[3], const int hi[3]) {
  if (!g || g->assembled) return g ? SSAMG_ERR_STATE : SSAMG_ERR_ARG;
  if (part < 0 || part >= g->nparts || !lo || !hi) return SSAMG_ERR_ARG;
  for (int d = 0; d < 3; ++d) {
    if (hi[d] < lo[d]) return SSAMG_ERR_ARG;
    if (d >= g->ndim && hi[d] != lo[d]) return SSAMG_ERR_ARG;
  }
  long long n = 1;
  for (int d = 0; d < 3; ++d) n *= (long long)hi[d] - lo[d] + 1;
  if (n > (1ll << 30)) return SSAMG_ERR_UNSUPPORTED;
  for (int d = 0; d < 3; ++d) {
    g->lo[part][d] = lo[d];
    g->hi[part][d] = hi[d];
  }
  g->set[part] = 1;
  g->boxes[part].clear();
  return SSAMG_OK;
}

extern "C" int ssamg_grid_add_box(ssamg_grid g, int part, const int lo[3], const int hi[3]) {
  if (!g || g->assembled) return g ? SSAMG_ERR_STATE : SSAMG_ERR_ARG;
  if (part < 0 || part >= g->nparts || !lo || !hi || !g->set[part]) return SSAMG_ERR_ARG;
  if ((int)g->boxes[part].size() >= SSAMG_MAX_PART_BOXES) return SSAMG_ERR_UNSUPPORTED;
  for (int d = 0; d < 3; ++d) {
    if (hi[d] < lo[d]) return SSAMG_ERR_ARG;
    if (d >= g->ndim && (lo[d] != g->lo[part][d] || hi[d] != g->hi[part][d])) return SSAMG_ERR_ARG;
  }
  std::array<int, 3> nlo = g->lo[part], nhi = g->hi[part];
  for (int d = 0; d < 3; ++d) {
    nlo[d] = std::min(nlo[d], lo[d]);
    nhi[d] = std::max(nhi[d], hi[d]);
  }
  long long n = 1;
  for (int d = 0; d < 3; ++d) n *= (long long)nhi[d] - nlo[d] + 1;
  if (n > (1ll << 30)) return SSAMG_ERR_UNSUPPORTED;
  if (g->boxes[part].empty())  // the box given by set_box is the first
    g->boxes[part].push_back({g->lo[part][0], g->lo[part][1], g->lo[part][2], g->hi[part][0],
                              g->hi[part][1], g->hi[part][2]});
  g->boxes[part].push_back({lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]});
  g->lo[part] = nlo;
  g->hi[part] = nhi;
  return SSAMG_OK;
}

extern "C" int ssamg_grid_assemble(ssamg_grid g) {
  if (!g) return SSAMG_ERR_ARG;
  for (int p = 0; p < g->nparts; ++p)
    if (!g->set[p]) return SSAMG_ERR_ARG;
  g->off.assign(g->nparts + 1, 0);
  for (int p = 0; p < g->nparts; ++p) g->off[p + 1] = g->off[p] + g->ncell(p);
  if (g->off.back() >= (1ll << 31)) return SSAMG_ERR_UNSUPPORTED;
  g->N = g->off.back();
  g->assembled = true;
  return SSAMG_OK;
}

extern "C" long long ssamg_grid_num_cells(ssamg_grid g) {
  return (g && g->assembled) ? g->N : -1;
}

extern "C" void ssamg_grid_destroy(ssamg_grid g) { delete g; }

// ---------------------------------------------------------------------------
// Matrix
// ---------------------------------------------------------------------------
extern "C" int ssamg_matrix_create(ssamg_grid g, int nentries, const int* offsets,
                                   ssamg_matrix* out) {
  if (!g || !out || !offsets || nentries < 1 || nentries > SSAMG_MAXE) return SSAMG_ERR_ARG;
  if (!g->assembled) return SSAMG_ERR_STATE;
  for (int e = 0; e < nentries; ++e) {
    for (int d = 0; d < 3; ++d) {
      int v = offsets[3 * e + d];
      if (v < -1 || v > 1) return SSAMG_ERR_ARG;
      if (d >= g->ndim && v != 0) return SSAMG_ERR_ARG;
    }
    for (int f = 0; f < e; ++f)
      if (offsets[3 * f] == offsets[3 * e] && offsets[3 * f + 1] == offsets[3 * e + 1] &&
          offsets[3 * f + 2] == offsets[3 * e + 2])
        return SSAMG_ERR_ARG;
  }
  auto* A = new (std::nothrow) ssamg_matrix_s;
  if (!A) return SSAMG_ERR_OOM;
  A->g = g;
  A->nent = nentries;
  for (int e = 0; e < nentries; ++e)
    for (int d = 0; d < 3; ++d) A->o[e][d] = offsets[3 * e + d];
  A->cval.assign(g->nparts, std::vector<double>(nentries, 0.0));
  A->tmpvar.assign(g->nparts, std::vector<double*>(nentries, nullptr));
  A->isset.assign(g->nparts, std::vector<char>(nentries, 0));
  A->isvar.assign(g->nparts, std::vector<char>(nentries, 0));
  *out = A;
  return SSAMG_OK;
}

extern "C" int ssamg_matrix_set_constant(ssamg_matrix A, int part, int entry, double value) {
  if (!A || part < 0 || part >= A->g->nparts || entry < 0 || entry >= A->nent) return SSAMG_ERR_ARG;
  if (A->tmpvar[part][entry]) {
    pool_fence();
    pool_free(A->tmpvar[part][entry]);
    A->tmpvar[part][entry] = nullptr;
  }
  A->cval[part][entry] = value;
  A->isvar[part][entry] = 0;
  A->isset[part][entry] = 1;
  A->assembled = false;
  return SSAMG_OK;
}

extern "C" int ssamg_matrix_set_box_values(ssamg_matrix A, int part, int entry, const double* vals,
                                           int vals_on_device) {
  if (!A || !vals || part < 0 || part >= A->g->nparts || entry < 0 || entry >= A->nent)
    return SSAMG_ERR_ARG;
  long long n = A->g->ncell(part);
  double*& dst = A->tmpvar[part][entry];
  if (!dst && !(dst = (double*)pool_alloc(sizeof(double) * n))) return SSAMG_ERR_OOM;
  cudaError_t e = cudaMemcpy(dst, vals, sizeof(double) * n,
                             vals_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    g_last_error = cudaGetErrorString(e);
    return SSAMG_ERR_CUDA;
  }
  A->isvar[part][entry] = 1;
  A->isset[part][entry] = 1;
  A->assembled = false;
  return SSAMG_OK;
}

extern "C" int ssamg_matrix_add_couplings(ssamg_matrix A, long long n, const int* part,
                                          const int* idx, const int* dir, const int* nbor_part,
                                          const int* nbor_idx, const double* vals) {
  if (!A || n < 0) return SSAMG_ERR_ARG;
  if (n == 0) return SSAMG_OK;
  if (!part || !idx || !dir || !nbor_part || !nbor_idx || !vals) return SSAMG_ERR_ARG;
  const ssamg_grid g = A->g;
  const int np = g->nparts;
  // validated and converted in one pass into the tail; a rejected call
  // leaves the matrix as it was
  const size_t m0 = A->c_val.size();
  A->c_row.resize(m0 + n);
  A->c_col.resize(m0 + n);
  A->c_bits.resize(m0 + n);
  A->c_val.resize(m0 + n);
  std::vector<char> hasu(A->c_hasu);
  hasu.resize(np, 0);
  // the parts' boxes and first cells in local arrays (the loop's stores do
  // not alias them)
  std::vector<int> lo(3 * np), hi(3 * np);
  std::vector<long long> off(np);
  for (int p = 0; p < np; ++p) {
    for (int d = 0; d < 3; ++d) {
      lo[3 * p + d] = g->lo[p][d];
      hi[3 * p + d] = g->hi[p][d];
    }
    off[p] = g->off[p];
  }
  const int ndim = g->ndim;
  const int* LO = lo.data();
  const int* HI = hi.data();
  const long long* OFF = off.data();
  int* crow = A->c_row.data() + m0;
  int* ccol = A->c_col.data() + m0;
  unsigned char* cbits = A->c_bits.data() + m0;
  double* cval = A->c_val.data() + m0;
  auto gidx = [&](int p, const int* c) {
    const int* l = LO + 3 * p;
    const int* h = HI + 3 * p;
    const long long nx = h[0] - l[0] + 1, ny = h[1] - l[1] + 1;
    return OFF[p] + ((long long)(c[2] - l[2]) * ny + (c[1] - l[1])) * nx + (c[0] - l[0]);
  };
  // One chunk of couplings [t0, t1): converts them into the tail and raises
  // its own part flags in hu; false at the first invalid coupling.
  auto convert = [&](long long t0, long long t1, char* hu) {
    for (long long t = t0; t < t1; ++t) {
      const int p = part[t], q = nbor_part[t];
      if (p < 0 || p >= np || q < 0 || q >= np || p == q) return false;
      const int* a = idx + 3 * t;
      const int* b = nbor_idx + 3 * t;
      const int* dv = dir + 3 * t;
      const int* lp = LO + 3 * p;
      const int* hp = HI + 3 * p;
      const int* lq = LO + 3 * q;
      const int* hq = HI + 3 * q;
      unsigned bt = 0;
      bool face = false, bad = false;
      for (int d = 0; d < 3; ++d) {
        bad |= a[d] < lp[d] || a[d] > hp[d] || b[d] < lq[d] || b[d] > hq[d] || dv[d] < -1 ||
               dv[d] > 1;
        bt |= (dv[d] > 0 ? 1u << (2 * d) : 0u) | (dv[d] < 0 ? 1u << (2 * d + 1) : 0u);
        face |= d < ndim && (a[d] == lp[d] || a[d] == hp[d]);
      }
      if (!bad) {
        // a nonzero direction leaves the row's part: the neighbour that way
        // lies outside its box, or outside the boxes of a part of several
        for (int d = 0; d < 3 && !bad; ++d) {
          if (dv[d] == 0) continue;
          int nb[3] = {a[0], a[1], a[2]};
          nb[d] += dv[d];
          bad = g->in_box(p, nb) && g->in_part(p, nb);
        }
        bad = bad || !g->in_part(p, a) || !g->in_part(q, b);
      }
      if (bad) return false;
      crow[t] = (int)gidx(p, a);
      ccol[t] = (int)gidx(q, b);
      cbits[t] = (unsigned char)bt;
      cval[t] = vals[t];
      // 2 when a row lies inside the box (no face of an active dimension)
      const char hv = face ? 1 : 2;
      if (hu[p] < hv) hu[p] = hv;
    }
    return true;
  };
  // large calls in chunks on host threads (every coupling is written by one
  // thread; the part flags are merged by maximum, so the result does not
  // depend on the split)
  const long long chunk = 16384;
  const int nth = (int)std::max<long long>(
      1, std::min<long long>({(long long)std::max(1u, std::thread::hardware_concurrency()),
                              (long long)SSAMG_HOST_THREADS, n / chunk}));
  bool ok = true;
  if (nth == 1) {
    ok = convert(0, n, hasu.data());
  } else {
    std::vector<std::vector<char>> hus(nth, std::vector<char>(np, 0));
    std::vector<char> oks(nth, 1);
    std::vector<std::thread> th;
    th.reserve(nth);
    for (int i = 0; i < nth; ++i)
      th.emplace_back([&, i] {
        oks[i] = convert(n * i / nth, n * (i + 1) / nth, hus[i].data());
      });
    for (auto& t : th) t.join();
    for (int i = 0; i < nth; ++i) {
      ok = ok && oks[i];
      for (int p = 0; p < np; ++p) hasu[p] = std::max(hasu[p], hus[i][p]);
    }
  }
  if (!ok) {
    A->c_row.resize(m0);
    A->c_col.resize(m0);
    A->c_bits.resize(m0);
    A->c_val.resize(m0);
    return SSAMG_ERR_ARG;
  }
  A->c_hasu.swap(hasu);
  A->assembled = false;
  return SSAMG_OK;
}

// Order in which a matrix's stencil entries are stored and, on level 0,
// held by the solver: offset-code order ((ox+1) + 3 (oy+1) + 9 (oz+1)) for a
// full 27-point stencil (whose specialised kernels expect it), else the
// user's entry order.
std::vector<int> storage_order(const ssamg_matrix_s* A) {
  std::vector<int> order(A->nent);
  for (int e = 0; e < A->nent; ++e) order[e] = e;
  if (A->nent == 27)
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      auto code = [&](int e) { return (A->o[e][0] + 1) + 3 * (A->o[e][1] + 1) + 9 * (A->o[e][2] + 1); };
      return code(a) < code(b);
    });
  return order;
}

extern "C" int ssamg_matrix_assemble(ssamg_matrix A, void* stream) {
  if (!A) return SSAMG_ERR_ARG;
  NvtxRange nv("ssamg_matrix_assemble");
  cudaStream_t st = (cudaStream_t)stream;
  API_BEGIN
  const ssamg_grid g = A->g;
  const int np = g->nparts;
  for (int p = 0; p < np; ++p)
    for (int e = 0; e < A->nent; ++e)
      argcheck(A->isset[p][e], "every stencil entry of every part needs a value");
  A->free_device();
  // a part of several boxes: every entry per cell over the bounding box (the
  // constants spread), masked below
  for (int p = 0; p < np; ++p) {
    if (g->boxes[p].empty()) continue;
    for (int e = 0; e < A->nent; ++e)
      if (!A->isvar[p][e]) {
        double*& dst = A->tmpvar[p][e];
        if (!dst && !(dst = (double*)pool_alloc(sizeof(double) * g->ncell(p))))
          throw SsamgError{SSAMG_ERR_OOM, "device allocation failed"};
        launch_fill(dst, g->ncell(p), A->cval[p][e], st);
        A->isvar[p][e] = 1;
      }
  }
  // pack variable entries (a 27-point stencil in offset-code order, so that
  // a part with every entry per cell is one contiguous array in that order)
  A->coef_off.assign(np, std::vector<long long>(A->nent, -1));
  const std::vector<int> order = storage_order(A);
  long long n = 0;
  for (int p = 0; p < np; ++p)
    for (int e : order)
      if (A->isvar[p][e]) {
        A->coef_off[p][e] = n;
        n += g->ncell(p);
      }
  A->ncoef = n;
  A->coef = pool_new<double>(n);
  for (int p = 0; p < np; ++p)
    for (int e = 0; e < A->nent; ++e)
      if (A->isvar[p][e]) {
        SSAMG_CUDA(cudaMemcpyAsync(A->coef + A->coef_off[p][e], A->tmpvar[p][e],
                                   sizeof(double) * g->ncell(p), cudaMemcpyDeviceToDevice, st));
        // S has no connection that leaves the box: store exact zeros there
        int ext[3] = {g->hi[p][0] - g->lo[p][0] + 1, g->hi[p][1] - g->lo[p][1] + 1,
                      g->hi[p][2] - g->lo[p][2] + 1};
        if (A->o[e][0] || A->o[e][1] || A->o[e][2])
          launch_mask_outside(A->coef + A->coef_off[p][e], ext, A->o[e], st);
        if (!g->boxes[p].empty()) {
          // cells outside the part's boxes: decoupled (diagonal 1), and no
          // connection into them
          PartBoxes pb{};
          pb.n = (int)g->boxes[p].size();
          for (int b = 0; b < pb.n; ++b)
            for (int t = 0; t < 6; ++t)
              pb.b[b][t] = g->boxes[p][b][t] - g->lo[p][t % 3];
          launch_mask_part(A->coef + A->coef_off[p][e], ext, A->o[e], pb, st);
        }
      }
  // couplings: global (row, col) and direction bits per coupling here,
  // O(m); the CSR (rows ascending, columns ascending, duplicates summed in
  // input order) on the device
  const long long m = (long long)A->c_val.size();
  A->has_u.assign(np, 0);
  for (int p = 0; p < np && p < (int)A->c_hasu.size(); ++p) A->has_u[p] = A->c_hasu[p];
  A->nr = 0;
  A->nnz = 0;
  if (m > 0) {
    int* drow = pool_new<int>(m);
    int* dcol = pool_new<int>(m);
    double* dval = pool_new<double>(m);
    unsigned char* dbits = pool_new<unsigned char>(m);
    SSAMG_CUDA(cudaMemcpyAsync(drow, A->c_row.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st));
    SSAMG_CUDA(cudaMemcpyAsync(dcol, A->c_col.data(), sizeof(int) * m, cudaMemcpyHostToDevice, st));
    SSAMG_CUDA(cudaMemcpyAsync(dval, A->c_val.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
    SSAMG_CUDA(cudaMemcpyAsync(dbits, A->c_bits.data(), m, cudaMemcpyHostToDevice, st));
    // outputs sized by the bound m (the row and entry counts come back below)
    A->u_rows = pool_new<int>(m);
    A->u_ptr = pool_new<int>(m + 1);
    A->u_col = pool_new<int>(m);
    A->u_val = pool_new<double>(m);
    A->u_bits = pool_new<unsigned char>(m);
    A->u_map = pool_new<int>(g->N);
    UAssemble ua{(int)g->N, m, drow, dcol, dval, dbits, A->u_rows, A->u_ptr,
                 A->u_col, A->u_val, A->u_bits, A->u_map};
    launch_uassemble(ua, &A->nr, &A->nnz, st);  // synchronises st
    for (void* q : {(void*)drow, (void*)dcol, (void*)dval, (void*)dbits}) pool_free(q);
  }
  SSAMG_CUDA(cudaStreamSynchronize(st));
  A->assembled = true;
  A->version++;
  return SSAMG_OK;
  API_END
}

extern "C" void ssamg_matrix_destroy(ssamg_matrix A) { delete A; }

// ---------------------------------------------------------------------------
// Solver: parameters
// ---------------------------------------------------------------------------
extern "C" void ssamg_params_default(ssamg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->precision = 0;
  p->relax = 0;
  p->relax_factor = 0.0;
  p->skip = 0;
  p->max_levels = 64;
  p->s_max = 0;
  p->tol = 1e-8;
  p->max_iter = 200;
  p->coarse_direct = 1;
  p->flexible = 0;
  p->use_graph = 1;
  p->use_tail = 3;
  p->use_pdl = 1;
  p->tail_cells = 0;
  p->use_bricks = 1;
  p->rhs_together = 1;
}

extern "C" int ssamg_solver_create(const ssamg_params* prm, ssamg_solver* out) {
  if (!prm || !out) return SSAMG_ERR_ARG;
  if (prm->precision < 0 || prm->precision > 1 || prm->relax < 0 || prm->relax > 1 ||
      prm->skip < 0 || prm->skip > 2 || prm->max_levels < 1 || prm->tol < 0 || prm->max_iter < 0 ||
      prm->use_tail < 0 || prm->use_tail > 3 || prm->rhs_together < 0 || prm->rhs_together > 1)
    return SSAMG_ERR_ARG;
  auto* s = new (std::nothrow) ssamg_solver_s;
  if (!s) return SSAMG_ERR_OOM;
  s->prm = *prm;
  *out = s;
  return SSAMG_OK;
}

extern "C" void ssamg_solver_destroy(ssamg_solver s) { delete s; }

// ---------------------------------------------------------------------------
// Setup
// ---------------------------------------------------------------------------
namespace {

int choose_direction(const double* Wp, const int* ext, int ndim) {
  // argmin_d W_pd over dimensions with extent > 1; ties -> smallest index
  int best = -1;
  for (int d = 0; d < ndim; ++d)
    if (ext[d] > 1 && (best < 0 || Wp[d] < Wp[best])) best = d;
  if (best < 0) {
    best = 0;
    for (int d = 1; d < ndim; ++d)
      if (Wp[d] < Wp[best]) best = d;
  }
  return best;
}

double relaxation_weight(const double* Wp, int dstar, int ndim) {
  // omega_p = 2 / (3 - beta_p / alpha_p) (Eqs. relax1, alpha-beta)
  double alpha = 0, inv_d = 0;
  for (int d = 0; d < ndim; ++d) {
    double v = std::isfinite(Wp[d]) ? 1.0 / (Wp[d] * Wp[d]) : 0.0;
    alpha += v;
    if (d == dstar) inv_d = v;
  }
  if (alpha <= 0.0) return 1.0;
  return 2.0 / (3.0 - (alpha - inv_d) / alpha);
}

void fill_dpart(DPart& dp, const PartH& h) {
  std::memset(&dp, 0, sizeof(dp));
  for (int d = 0; d < 3; ++d) dp.n[d] = h.n[d];
  dp.ncell = (int)h.ncell;
  dp.off = h.off;
  dp.nent = h.nent;
  dp.dstar = h.dstar;
  dp.par = h.par;
  dp.omega = h.omega;
  dp.has_u = h.has_u;
  dp.skip = h.skip;
  dp.dx = make_fastdiv(h.n[0]);
  dp.dxy = make_fastdiv(h.n[0] * h.n[1]);
  std::memset(dp.slot, -1, sizeof(dp.slot));
  for (int e = 0; e < h.nent; ++e) {
    for (int d = 0; d < 3; ++d) dp.o[e][d] = (signed char)h.o[e][d];
    dp.disp[e] = h.o[e][0] + h.o[e][1] * h.n[0] + h.o[e][2] * h.n[0] * h.n[1];
    dp.coef[e] = h.var[e] ? h.coef_off[e] : -1;
    dp.cval[e] = h.cval[e];
    dp.cval32[e] = (float)h.cval[e];
    dp.slot[(h.o[e][0] + 1) + 3 * (h.o[e][1] + 1) + 9 * (h.o[e][2] + 1)] = (signed char)e;
    dp.uent[e] = (signed char)h.uent[e];
  }
  dp.allvar = 1;
  dp.varmask = 0;
  for (int e = 0; e < h.nent; ++e) {
    if (h.var[e]) dp.varmask |= 1u << e;
    if (!h.var[e] || h.coef_off[e] != h.coef_off[0] + (long long)e * h.ncell) dp.allvar = 0;
  }
  dp.zeroext = dp.allvar;
  dp.canon27 = h.nent == 27;
  for (int e = 0; e < h.nent && dp.canon27; ++e)
    if ((h.o[e][0] + 1) + 3 * (h.o[e][1] + 1) + 9 * (h.o[e][2] + 1) != e) dp.canon27 = 0;
  for (int d = 0; d < 3; ++d) dp.nf[d] = h.nf[d];
  dp.nfine = (int)h.nfine;
  dp.poff = h.poff;
  dp.fdx = make_fastdiv(std::max(1, h.nf[0]));
  dp.fdxy = make_fastdiv(std::max(1, h.nf[0] * h.nf[1]));
}

// A vector of n elements of w bytes with `guard` zeroed elements before and
// after it (stencils on levels whose coefficients vanish outside the box read
// up to one plane past either end without bounds tests).
void* padded_vector(ssamg_solver s, size_t w, long long n, long long guard, cudaStream_t st) {
  char* base = (char*)s->arena.alloc(w * (size_t)(n + 2 * guard));
  SSAMG_CUDA(cudaMemsetAsync(base, 0, w * (size_t)(n + 2 * guard), st));
  return base + w * guard;
}

// Size class of a level of n cells in the tile table: floor(log2(max(n, 1))).
int tile_class(long long n) {
  int c = 0;
  while (c < SSAMG_TILE_CLASSES - 1 && (2ll << c) <= n) ++c;
  return c;
}

long long level_cells(const Level& L) {
  long long n = 0;
  for (const PartH& h : L.parts) n += h.ncell;
  return n;
}

bool valid_tile(int t) {
  const int k = t & ~SSAMG_TILE_BRICKS;
  return t == 0 || (k >= 1 && k <= SSAMG_CPT_LARGE);
}

// Block starts of a level's launches and the first cell of every part (host
// side of the level's device tables).
struct LevelTables {
  std::vector<int> blk, bblk, fblk, cs;
};

// The host side of a level's tables: part descriptors (L.dparts), tile and
// brick decomposition, operator-apply shape.  Copies nothing.
void level_tables(ssamg_solver s, Level& L, const Level* next, LevelTables& t) {
  const int np = L.np;
  L.dparts.assign(np, DPart{});
  std::vector<int>& blk = t.blk;
  std::vector<int>& fblk = t.fblk;
  std::vector<int>& cs = t.cs;
  blk.assign(np + 1, 0);
  fblk.assign(np + 1, 0);
  cs.assign(np + 1, 0);
  const long long ntot = level_cells(L);
  // tile form: the table's entry for the level's size class, else the
  // built-in rule (SSAMG_CPT_LARGE cells per thread on large levels)
  const int te = s->tiles[tile_class(ntot)];
  L.cpt = te ? (te & ~SSAMG_TILE_BRICKS) : ntot >= SSAMG_CPT_MIN_CELLS ? SSAMG_CPT_LARGE : 1;
  L.bricks = te ? (te & SSAMG_TILE_BRICKS) != 0 : 1;
  const long long tile = (long long)L.cpt * SSAMG_BLOCK;
  for (int p = 0; p < np; ++p) {
    const PartH& h = L.parts[p];
    blk[p + 1] = blk[p] + (int)cdivll(h.ncell, tile);
    fblk[p + 1] = fblk[p] + (int)cdivll(h.nfine, tile);
    cs[p + 1] = cs[p] + (int)h.ncell;
  }
  L.nblk = blk[np];
  L.nfblk = fblk[np];
  // bricks (checked 7-point operator applies)
  std::vector<int>& bblk = t.bblk;
  bblk.assign(np + 1, 0);
  for (int p = 0; p < np; ++p) {
    const PartH& h = L.parts[p];
    const long long nb = cdivll(h.n[0], SSAMG_BRICK_X) * cdivll(h.n[1], SSAMG_BRICK_Y) *
                         cdivll(h.n[2], SSAMG_BRICK_Z);
    bblk[p + 1] = bblk[p] + (int)nb;
  }
  L.nbblk = bblk[np];
  L.brick_fill = L.nbblk ? (double)ntot / ((double)L.nbblk * SSAMG_BRICK_X * SSAMG_BRICK_Y *
                                           SSAMG_BRICK_Z)
                         : 0.0;
  L.hbblk = bblk;
  L.hblk = blk;
  for (int p = 0; p < np; ++p) {
    DPart& dp = L.dparts[p];
    fill_dpart(dp, L.parts[p]);
    dp.prob = s->part_prob.empty() ? 0 : s->part_prob[p];
    dp.blk0 = blk[p];
    dp.fblk0 = fblk[p];
    dp.bblk0 = bblk[p];
    dp.bb[0] = (int)cdivll(L.parts[p].n[0], SSAMG_BRICK_X);
    dp.bb[1] = (int)cdivll(L.parts[p].n[1], SSAMG_BRICK_Y);
    dp.bb[2] = (int)cdivll(L.parts[p].n[2], SSAMG_BRICK_Z);
    dp.cpt = L.cpt;
    if (next) {
      const PartH& c = next->parts[p];
      dp.coff = c.off;
      for (int d = 0; d < 3; ++d) dp.cn[d] = c.n[d];
      dp.cncell = (int)c.ncell;
      dp.cdx = make_fastdiv(c.n[0]);
      dp.cdxy = make_fastdiv(c.n[0] * c.n[1]);
    }
  }
  {
    // operator-apply shape shared by all parts (see StencilShape)
    bool unchecked = true, all27 = true, all7 = true, all15 = true, canon7 = true;
    static const int c7[7][3] = {{0, 0, 0}, {-1, 0, 0}, {1, 0, 0}, {0, -1, 0},
                                 {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (const DPart& dp : L.dparts) {
      unchecked = unchecked && dp.allvar && dp.zeroext;
      all27 = all27 && dp.canon27;
      all7 = all7 && dp.nent == 7;
      all15 = all15 && dp.nent == 15;
      if (dp.nent != 7) canon7 = false;
      for (int e = 0; e < 7 && canon7; ++e)
        for (int d = 0; d < 3; ++d)
          if (dp.o[e][d] != c7[e][d]) canon7 = false;
    }
    L.shape = !unchecked ? (canon7 ? 5 : 0) : all27 ? 3 : all7 ? 1 : all15 ? 2 : 4;
    L.kvar = 0;
    for (const DPart& dp : L.dparts)
      L.kvar = std::max(L.kvar, dp.varmask == 0 ? 0 : dp.varmask == 1u ? 1 : 2);
  }
}

// One level's tables, copied on their own (level 0 before the coupling sums,
// and a level whose coupling rows vanished).  The copies are from pageable
// memory, so they are done when the call returns.
void upload_level(ssamg_solver s, Level& L, const Level* next, cudaStream_t st) {
  LevelTables t;
  level_tables(s, L, next, t);
  const int np = L.np;
  if (!L.d_parts) {
    L.d_parts = aalloc<DPart>(s->arena, np);
    L.d_blk = aalloc<int>(s->arena, np + 1);
    L.d_bblk = aalloc<int>(s->arena, np + 1);
    L.d_fblk = aalloc<int>(s->arena, np + 1);
    L.d_cellstart = aalloc<int>(s->arena, np + 1);
  }
  SSAMG_CUDA(cudaMemcpyAsync(L.d_parts, L.dparts.data(), sizeof(DPart) * np, cudaMemcpyHostToDevice, st));
  SSAMG_CUDA(cudaMemcpyAsync(L.d_blk, t.blk.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice, st));
  SSAMG_CUDA(cudaMemcpyAsync(L.d_bblk, t.bblk.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice, st));
  SSAMG_CUDA(cudaMemcpyAsync(L.d_fblk, t.fblk.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice, st));
  SSAMG_CUDA(cudaMemcpyAsync(L.d_cellstart, t.cs.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice, st));
}

// Every level's tables in one device block, through one pinned staging
// buffer and one copy.  The buffer is reused by the next set-up, which
// starts after this one has synchronised the stream.
void upload_levels(ssamg_solver s, cudaStream_t st) {
  const int nl = (int)s->lev.size();
  std::vector<LevelTables> t(nl);
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t total = 0;
  for (int l = 0; l < nl; ++l) {
    level_tables(s, s->lev[l], l + 1 < nl ? &s->lev[l + 1] : nullptr, t[l]);
    const size_t np = (size_t)s->lev[l].np;
    total += al(sizeof(DPart) * np) + 4 * al(sizeof(int) * (np + 1));
  }
  if (s->h_up_cap < total) {
    pinned_free(s->h_up);
    s->h_up = nullptr;
    s->h_up_cap = 0;
    s->h_up = pinned_new<char>((long long)total);
    s->h_up_cap = total;
  }
  char* dev = (char*)s->arena.alloc(total);
  size_t o = 0;
  auto put = [&](const void* src, size_t bytes) {
    std::memcpy(s->h_up + o, src, bytes);
    void* d = dev + o;
    o += al(bytes);
    return d;
  };
  for (int l = 0; l < nl; ++l) {
    Level& L = s->lev[l];
    const size_t np = (size_t)L.np;
    L.d_parts = (DPart*)put(L.dparts.data(), sizeof(DPart) * np);
    L.d_blk = (int*)put(t[l].blk.data(), sizeof(int) * (np + 1));
    L.d_bblk = (int*)put(t[l].bblk.data(), sizeof(int) * (np + 1));
    L.d_fblk = (int*)put(t[l].fblk.data(), sizeof(int) * (np + 1));
    L.d_cellstart = (int*)put(t[l].cs.data(), sizeof(int) * (np + 1));
  }
  SSAMG_CUDA(cudaMemcpyAsync(dev, s->h_up, o, cudaMemcpyHostToDevice, st));
}

// Coarse-level transition run by one cluster (see kernels_tail.cu): picks the
// first tail level (the first level of at most tail_cells cells whose tail
// fits the cluster's shared memory), lays out the per-CTA images, and
// assembles them.  Leaves s->ctail_lt = -1 when no tail of two or more levels
// fits or the device cannot run the cluster.  Synchronises st.
void build_ctail(ssamg_solver s, cudaStream_t st) {
  s->ctail_lt = -1;
  const int Lc = (int)s->lev.size() - 1;
  const bool fp32 = s->prm.precision == 1;
  const bool direct = s->prm.coarse_direct != 0;
  if (Lc < 1 || (direct && !s->cinv)) return;
  const long long maxc = s->prm.tail_cells > 0 ? s->prm.tail_cells : SSAMG_CTAIL_CELLS;
  int lt = Lc;
  while (lt - 1 >= 1 && s->lev[lt - 1].N <= maxc) --lt;
  if (lt >= Lc) return;
  int dev = 0, optin = 0;
  SSAMG_CUDA(cudaGetDevice(&dev));
  SSAMG_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // row lengths of every candidate level (one read-back)
  std::vector<long long> first(Lc + 2, 0);
  for (int l = lt; l <= Lc; ++l) first[l + 1] = first[l] + s->lev[l].N;
  int* dlen = aalloc<int>(s->arena, first[Lc + 1] - first[lt]);
  {
    std::vector<int*> lens;
    for (int l = lt; l <= Lc; ++l) lens.push_back(dlen + (first[l] - first[lt]));
    launch_ctail_rowlen(s->lev, lt, Lc, lens.data(), st);
  }
  std::vector<int> len(first[Lc + 1] - first[lt]);
  SSAMG_CUDA(cudaMemcpyAsync(len.data(), dlen, sizeof(int) * len.size(), cudaMemcpyDeviceToHost, st));
  SSAMG_CUDA(cudaStreamSynchronize(st));
  const size_t w = fp32 ? sizeof(float) : sizeof(double);
  auto al = [](long long v) { return (v + 15) & ~15ll; };
  for (int nc : {SSAMG_CTAIL_MAX_CTAS, 8}) {
    for (int t0 = lt; t0 < Lc; ++t0) {
      const int nt = Lc - t0 + 1;
      if (nt > SSAMG_CTAIL_MAX_LEVELS) continue;
      CTailArgs a{};
      a.nt = nt;
      a.direct = direct;
      a.nL = (int)s->lev[Lc].N;
      long long vec = 0, ro = 0;
      bool ok = true;
      std::vector<long long> cap(nt);
      // row pointers of every level first, so that one 2-D copy uploads them
      for (int j = 0; j < nt; ++j) {
        a.lev[j].S = (int)cdivll(s->lev[t0 + j].N, nc);
        a.lev[j].o_rowptr = (int)ro;
        ro += 4ll * (a.lev[j].S + 1);
      }
      ro = al(ro);
      const long long rp_bytes = ro;
      for (int j = 0; j < nt && ok; ++j) {
        const Level& L = s->lev[t0 + j];
        CTailLevel& v = a.lev[j];
        v.n = (int)L.N;
        v.S = (int)cdivll(L.N, nc);
        // lanes per row: as many as leave every row of the slice a group in one pass
        v.tpr = 1;
        while (v.tpr < 32 && (long long)v.S * v.tpr * 2 <= SSAMG_CTAIL_THREADS) v.tpr *= 2;
        if (v.S >= (1 << SSAMG_CTAIL_LOCAL_BITS)) ok = false;
        long long mx = 0;
        for (int c = 0; c < nc; ++c) {
          long long sum = 0;
          for (long long g = (long long)c * v.S; g < std::min<long long>(L.N, (long long)(c + 1) * v.S); ++g)
            sum += len[first[t0 + j] - first[lt] + g];
          mx = std::max(mx, sum);
        }
        cap[j] = mx;
        v.o_x = (int)vec;  vec += al(v.S * w);
        v.o_b = (int)vec;  vec += al(v.S * w);
        v.o_r = (int)vec;  vec += al(v.S * w);
        v.o_col = (int)ro;    ro += al(2 * mx);
        v.o_val = (int)ro;    ro += al(w * mx);
        v.o_dinv = (int)ro;   ro += al(w * v.S);
        v.o_pcol = v.o_pval = v.o_rcol = v.o_rval = v.o_inv = 0;
        if (j + 1 < nt) {
          v.o_pcol = (int)ro; ro += al(2ll * 2 * v.S);
          v.o_pval = (int)ro; ro += al(w * 2 * v.S);
        }
        if (j > 0) {
          v.o_rcol = (int)ro; ro += al(2ll * 3 * v.S);
          v.o_rval = (int)ro; ro += al(w * 3 * v.S);
        }
        if (j + 1 == nt && direct) {
          v.o_inv = (int)ro; ro += al(8ll * v.S * a.nL);
        }
      }
      if (!ok || vec + ro > optin) continue;
      a.vec_bytes = (int)vec;
      a.ro_bytes = ro;
      const bool can = fp32 ? ctail_prepare<float>(nc, vec + ro) : ctail_prepare<double>(nc, vec + ro);
      if (!can) break;  // try fewer CTAs
      // images: zeroed, row pointers from the host, the rest by the fill kernels
      char* img = (char*)s->arena.alloc((size_t)nc * ro);
      SSAMG_CUDA(cudaMemsetAsync(img, 0, (size_t)nc * ro, st));
      std::vector<int> rp((size_t)nc * rp_bytes / 4, 0);
      for (int j = 0; j < nt; ++j) {
        const CTailLevel& v = a.lev[j];
        for (int c = 0; c < nc; ++c) {
          int* row = rp.data() + ((size_t)c * rp_bytes + v.o_rowptr) / 4;
          int acc = 0;
          for (int li = 0; li < v.S; ++li) {
            row[li] = acc;
            const long long g = (long long)c * v.S + li;
            if (g < v.n) acc += len[first[t0 + j] - first[lt] + g];
          }
          row[v.S] = acc;
        }
      }
      SSAMG_CUDA(cudaMemcpy2DAsync(img, (size_t)ro, rp.data(), (size_t)rp_bytes, (size_t)rp_bytes,
                                   nc, cudaMemcpyHostToDevice, st));
      launch_ctail_fill(fp32, s->lev, t0, a, direct ? s->cinv : nullptr, img, ro, st);
      SSAMG_CUDA(cudaStreamSynchronize(st));  // rp is a host temporary
      a.image = img;
      s->ctail = a;
      s->ctail_lt = t0;
      s->ctail_nc = nc;
      s->ctail_smem = vec + ro;
      return;
    }
  }
}

void build_hierarchy(ssamg_solver s, cudaStream_t st) {
  ssamg_matrix A = s->A;
  const ssamg_grid g = A->g;
  const int np = g->nparts;
  const int ndim = g->ndim;
  const bool fp32 = s->prm.precision == 1;
  s->ndim = ndim;
  s->arena.reset();
  s->graphs.reset();
  s->rhs = RhsSet{};
  s->lev.clear();
  s->lev.reserve((size_t)s->prm.max_levels + 1);
  s->ready = false;

  if (!s->part_prob.empty() && (int)s->part_prob.size() != np)
    throw SsamgError{SSAMG_ERR_ARG, "the problem map does not match the grid's parts"};
  if (s->h_cap < s->nprob) {
    pinned_free(s->h_sc);
    pinned_free(s->h_int);
    pinned_free(s->h_dbl);
    s->h_sc = nullptr;
    s->h_int = nullptr;
    s->h_dbl = nullptr;
    s->h_sc = pinned_new<PcgScalars>(s->nprob);
    s->h_int = pinned_new<int>(16);
    s->h_dbl = pinned_new<double>(2 * s->nprob + 16);
    s->h_cap = s->nprob;
  }

  // ---- level 0 from the matrix
  s->lev.emplace_back();
  Level& L0 = s->lev[0];
  L0.np = np;
  L0.N = g->N;
  L0.parts.resize(np);
  for (int p = 0; p < np; ++p) {
    PartH& h = L0.parts[p];
    std::memset(&h, 0, sizeof(h));
    for (int d = 0; d < 3; ++d) {
      h.lo[d] = g->lo[p][d];
      h.hi[d] = g->hi[p][d];
      h.n[d] = h.hi[d] - h.lo[d] + 1;
    }
    h.ncell = g->ncell(p);
    h.off = (int)g->off[p];
    h.dstar = -1;
    h.nent = A->nent;
    const std::vector<int> order = storage_order(A);
    for (int e = 0; e < A->nent; ++e) {
      const int u = order[e];  // the user's entry held as entry e
      for (int d = 0; d < 3; ++d) h.o[e][d] = A->o[u][d];
      h.var[e] = A->isvar[p][u];
      h.cval[e] = A->cval[p][u];
      h.coef_off[e] = A->coef_off[p][u];
      h.uent[e] = u;
    }
    h.has_u = A->has_u[p];
  }
  L0.coef = A->coef;
  L0.ncoef = A->ncoef;
  L0.nr = A->nr;
  L0.nnz = A->nnz;
  L0.u_rows = A->u_rows;
  L0.u_ptr = A->u_ptr;
  L0.u_col = A->u_col;
  L0.u_val = A->u_val;
  L0.u_bits = A->u_bits;
  L0.u_map = A->u_map;
  upload_level(s, L0, nullptr, st);

  // ---- Section 3.1: coupling sums c and spacings W (one sync)
  double* d_partial = aalloc<double>(s->arena, 3ll * L0.nblk);
  double* d_c = aalloc<double>(s->arena, 3ll * np);
  launch_wsum(L0, d_partial, d_c, st);
  s->c.assign(3 * np, 0.0);
  SSAMG_CUDA(cudaMemcpyAsync(s->c.data(), d_c, sizeof(double) * 3 * np, cudaMemcpyDeviceToHost, st));
  SSAMG_CUDA(cudaStreamSynchronize(st));
  s->W.assign(3 * np, HUGE_VAL);
  if (!s->user_W.empty()) {
    // representative grid spacings given by the user (Section 3.1), used
    // for coarsening instead of the ones from the coupling sums
    if ((int)s->user_W.size() != 3 * np)
      throw SsamgError{SSAMG_ERR_ARG, "the spacings do not match the grid's parts"};
    for (int p = 0; p < np; ++p)
      for (int d = 0; d < ndim; ++d) s->W[3 * p + d] = s->user_W[3 * p + d];
  } else {
    for (int p = 0; p < np; ++p) {
      double cmax = -HUGE_VAL;
      for (int d = 0; d < ndim; ++d) cmax = std::max(cmax, s->c[3 * p + d]);
      for (int d = 0; d < ndim; ++d)
        if (s->c[3 * p + d] > 0 && cmax > 0) s->W[3 * p + d] = std::sqrt(cmax / s->c[3 * p + d]);
    }
  }

  // ---- Algorithm 1 on the host: boxes, d* and omega per level
  long long s_max = s->prm.s_max > 0 ? s->prm.s_max : np;
  std::vector<double> W = s->W;
  for (;;) {
    Level& F = s->lev.back();
    long long total = 0;
    bool any_active = false;
    for (auto& h : F.parts) {
      total += h.ncell;
      if (h.ncell > 1) any_active = true;
    }
    bool last = total <= s_max || (int)s->lev.size() >= s->prm.max_levels || !any_active;
    for (int p = 0; p < np; ++p) {
      PartH& h = F.parts[p];
      int d = choose_direction(&W[3 * p], h.n, ndim);
      h.omega = relaxation_weight(&W[3 * p], d, ndim);
      h.dstar = (!last && h.ncell > 1) ? d : -1;
    }
    if (last) break;
    Level C;
    C.np = np;
    C.parts.resize(np);
    long long off = 0;
    for (int p = 0; p < np; ++p) {
      PartH& h = F.parts[p];
      PartH& c = C.parts[p];
      std::memset(&c, 0, sizeof(c));
      for (int d = 0; d < 3; ++d) {
        c.lo[d] = h.lo[d];
        c.hi[d] = h.hi[d];
      }
      c.has_u = h.has_u;
      c.dstar = -1;
      if (h.dstar >= 0) {
        int d = h.dstar;
        c.lo[d] = ceildiv2(h.lo[d]);
        c.hi[d] = floordiv2(h.hi[d]);
        W[3 * p + d] *= 2.0;
        h.par = h.lo[d] & 1;
        for (int q = 0; q < 3; ++q) h.nf[q] = h.n[q];
        h.nf[d] = (h.n[d] + h.par) >> 1;
        h.nfine = (long long)h.nf[0] * h.nf[1] * h.nf[2];
        // coarse stencil: fine offsets projected off d*, times {-1,0,1} along d*
        bool present[27] = {false};
        for (int e = 0; e < h.nent; ++e)
          for (int od = -1; od <= 1; ++od) {
            int o[3] = {h.o[e][0], h.o[e][1], h.o[e][2]};
            o[d] = od;
            present[(o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1)] = true;
          }
        c.nent = 0;
        for (int code = 0; code < 27; ++code)
          if (present[code]) {
            c.o[c.nent][0] = code % 3 - 1;
            c.o[c.nent][1] = (code / 3) % 3 - 1;
            c.o[c.nent][2] = code / 9 - 1;
            ++c.nent;
          }
      } else {
        c.nent = h.nent;
        for (int e = 0; e < h.nent; ++e)
          for (int d = 0; d < 3; ++d) c.o[e][d] = h.o[e][d];
      }
      for (int d = 0; d < 3; ++d) c.n[d] = c.hi[d] - c.lo[d] + 1;
      c.ncell = (long long)c.n[0] * c.n[1] * c.n[2];
      c.off = (int)off;
      off += c.ncell;
      for (int e = 0; e < c.nent; ++e) {
        c.var[e] = 1;
        c.uent[e] = e;
      }
    }
    C.N = off;
    s->lev.push_back(std::move(C));
  }
  const int Lc = (int)s->lev.size() - 1;
  // "skip" (Section 3.4).  skip = 1: per part, the levels form rounds as
  // full coarsening would (a round starts at level 0 and at every level whose
  // d* already occurs in the current round; a level with no d* relaxes and
  // ends its round); only the first level of a round relaxes.  An isotropic
  // part (d*_l = d*_{l-n_d}) then relaxes on levels 0, n_d, 2 n_d, ...; a
  // part coarsened repeatedly along one direction relaxes on each of those
  // levels.  skip = 2: the printed test alone, no relaxation at l >= n_d
  // when d*_l = d*_{l-n_d}.
  for (int p = 0; p < np; ++p) {
    unsigned seen = 0;  // directions of the current round
    for (int l = 0; l <= Lc; ++l) {
      PartH& h = s->lev[l].parts[p];
      h.skip = 0;
      if (s->prm.skip == 2) {
        h.skip = l >= ndim && h.dstar >= 0 && h.dstar == s->lev[l - ndim].parts[p].dstar;
      } else if (s->prm.skip == 1) {
        if (h.dstar < 0) {
          seen = 0;
        } else if (seen == 0 || (seen >> h.dstar) & 1u) {
          seen = 1u << h.dstar;
        } else {
          seen |= 1u << h.dstar;
          h.skip = 1;
        }
      }
    }
  }

  // ---- allocation (one arena walk; identical sizes reuse the same memory)
  for (int l = 0; l <= Lc; ++l) {
    Level& L = s->lev[l];
    if (l > 0) {
      long long n = 0;
      for (auto& h : L.parts)
        for (int e = 0; e < h.nent; ++e) {
          h.coef_off[e] = n;
          n += h.ncell;
        }
      L.ncoef = n;
      L.coef = aalloc<double>(s->arena, n);
    }
    if (fp32) L.coef32 = aalloc<float>(s->arena, L.ncoef);
    long long nP = 0;
    for (auto& h : L.parts) {
      h.poff = (int)nP;
      nP += h.nfine;
    }
    L.nP = nP;
    if (l < Lc) {
      L.Pw = aalloc<double>(s->arena, nP);
      L.Pe = aalloc<double>(s->arena, nP);
      if (fp32) {
        L.Pw32 = aalloc<float>(s->arena, nP);
        L.Pe32 = aalloc<float>(s->arena, nP);
      }
    }
    L.dinv = aalloc<double>(s->arena, L.N);
    if (fp32) L.dinv32 = aalloc<float>(s->arena, L.N);
    L.guard = 0;
    for (auto& h : L.parts) L.guard = std::max<long long>(L.guard, 1 + h.n[0] + (long long)h.n[0] * h.n[1]);
    bool any_u = false;
    for (auto& h : L.parts) any_u |= h.has_u != 0;
    if (l > 0 && any_u) L.u_map = aalloc<int>(s->arena, L.N);
  }
  {
    // the cycle vectors x, b, r, t of every level (guard cells around each):
    // one zeroed block
    const size_t w = fp32 ? sizeof(float) : sizeof(double);
    auto vb = [&](const Level& L) { return (w * (size_t)(L.N + 2 * L.guard) + 255) & ~(size_t)255; };
    size_t total = 0;
    for (int l = 0; l <= Lc; ++l) total += 4 * vb(s->lev[l]);
    char* base = (char*)s->arena.alloc(total);
    SSAMG_CUDA(cudaMemsetAsync(base, 0, total, st));
    for (int l = 0; l <= Lc; ++l) {
      Level& L = s->lev[l];
      void** v[4] = {&L.x, &L.b, &L.r, &L.t};
      for (void** q : v) {
        *q = base + w * (size_t)L.guard;
        base += vb(L);
      }
    }
  }
  upload_levels(s, st);

  if (fp32) {
    launch_to_float(L0.coef, L0.coef32, L0.ncoef, st);
    if (L0.nnz > 0) {
      L0.u_val32 = aalloc<float>(s->arena, L0.nnz);
      launch_to_float(L0.u_val, L0.u_val32, L0.nnz, st);
    }
  }

  // ---- per level: P (Eq. prolEx), P^T S P and P^T U P (Eq. galerkin)
  long long maxN = 0;
  for (int l = 1; l <= Lc; ++l) maxN = std::max(maxN, s->lev[l].N);
  int* marker = nullptr;
  int* scan_tmp = nullptr;
  s->d_err = aalloc<int>(s->arena, 4);
  SSAMG_CUDA(cudaMemsetAsync(s->d_err, 0, sizeof(int) * 4, st));
  // The coupling rows of a coarse level are fixed by the structure alone
  // (which coarse cells the fine coupling rows' P rows reach), so they are
  // found one level ahead: each level waits on the host once, for the entry
  // count of its own U_c and the row count of the next level together.
  int* scan_tmp2 = nullptr;  // the side stream's scan scratch
  if (!s->ss) {
    SSAMG_CUDA(cudaStreamCreateWithFlags(&s->ss, cudaStreamNonBlocking));
    SSAMG_CUDA(cudaEventCreateWithFlags(&s->ev_p, cudaEventDisableTiming));
    SSAMG_CUDA(cudaEventCreateWithFlags(&s->ev_rap, cudaEventDisableTiming));
    SSAMG_CUDA(cudaEventCreateWithFlags(&s->ev_rows, cudaEventDisableTiming));
    SSAMG_CUDA(cudaEventCreateWithFlags(&s->ev_mark, cudaEventDisableTiming));
    SSAMG_CUDA(cudaEventCreateWithFlags(&s->ev_uc, cudaEventDisableTiming));
  }
  auto mark_rows = [&](const Level& F, const Level& C, cudaStream_t ms) {
    if (!marker) {
      marker = aalloc<int>(s->arena, maxN + 1);
      scan_tmp = aalloc<int>(s->arena, (long long)scan_tmp_ints(maxN + 1) + 1);
      scan_tmp2 = aalloc<int>(s->arena, (long long)scan_tmp_ints(maxN + 1) + 1);
    }
    launch_uprow(F, C, nullptr, nullptr, nullptr, marker, ms);
    launch_scan(marker, C.N, ms == st ? scan_tmp : scan_tmp2, ms);
  };
  auto make_rows = [&](Level& C, int nr) {
    C.nr = nr;
    C.u_rows = aalloc<int>(s->arena, C.nr);
    C.u_ptr = aalloc<int>(s->arena, C.nr + 1);
    launch_urows(C, marker, nullptr, st);
  };
  if (Lc > 0) {
    if (L0.nr > 0) {
      mark_rows(L0, s->lev[1], st);
      SSAMG_CUDA(cudaMemcpyAsync(s->h_int, marker + s->lev[1].N, sizeof(int),
                                 cudaMemcpyDeviceToHost, st));
      SSAMG_CUDA(cudaStreamSynchronize(st));
      make_rows(s->lev[1], s->h_int[0]);
      SSAMG_CUDA(cudaEventRecord(s->ev_rows, st));
    } else {
      s->lev[1].nr = 0;
    }
  }
  // Two kinds of work of a level run on a side stream beside the coupling
  // chain on st: the marking of the next level's coupling rows (it needs
  // only this coarse level's rows and the geometry; the host waits for its
  // row count through ev_mark) and the structured Galerkin product (it needs
  // only P, the interpolation just before it; the next level's
  // interpolation, which reads the coarse stencil, waits for it).
  // Level 0's operator is final already: its smoother diagonal (the largest
  // of them) runs on the side stream beside the whole level loop.
  SSAMG_CUDA(cudaEventRecord(s->ev_p, st));
  SSAMG_CUDA(cudaStreamWaitEvent(s->ss, s->ev_p, 0));
  launch_dinv(s->lev, 0, 0, s->prm.relax, s->prm.relax_factor, fp32, s->ss);
  for (int l = 0; l < Lc; ++l) {
    Level& F = s->lev[l];
    Level& C = s->lev[l + 1];
    Level* N2 = l + 2 <= Lc ? &s->lev[l + 2] : nullptr;
    NvtxRange nvl("ssamg setup level", l);
    const bool mark = N2 && F.nr > 0 && C.nr > 0;
    if (mark) {
      SSAMG_CUDA(cudaStreamWaitEvent(s->ss, s->ev_rows, 0));
      mark_rows(C, *N2, s->ss);
      SSAMG_CUDA(cudaMemcpyAsync(s->h_int + 1, marker + N2->N, sizeof(int),
                                 cudaMemcpyDeviceToHost, s->ss));
      SSAMG_CUDA(cudaEventRecord(s->ev_mark, s->ss));
    }
    if (l > 0) SSAMG_CUDA(cudaStreamWaitEvent(st, s->ev_rap, 0));
    launch_interp(F, fp32, st);
    SSAMG_CUDA(cudaEventRecord(s->ev_p, st));
    SSAMG_CUDA(cudaStreamWaitEvent(s->ss, s->ev_p, 0));
    if (F.nr > 0) {
      // P rows of the coupling columns (kept: the prolongation's row jobs
      // use them), on the side stream too; the merge waits for them
      F.u_pj = aalloc<int>(s->arena, 2 * F.nnz);
      F.u_pw = aalloc<double>(s->arena, 2 * F.nnz);
      if (fp32) F.u_pw32 = aalloc<float>(s->arena, 2 * F.nnz);
      launch_ucols(nullptr, F, fp32, true, false, s->ss);
      SSAMG_CUDA(cudaEventRecord(s->ev_uc, s->ss));
    }
    launch_rap_struct(F, C, fp32, s->ss);
    SSAMG_CUDA(cudaEventRecord(s->ev_rap, s->ss));
    C.nnz = 0;
    if (N2) N2->nr = 0;
    if (F.nr == 0) continue;
    if (C.nr == 0) continue;
    // P rows of the coupling rows, and the coarse rows they reach
    int* prI = aalloc<int>(s->arena, 2ll * F.nr);
    double* prW = aalloc<double>(s->arena, 2ll * F.nr);
    signed char* prA = aalloc<signed char>(s->arena, 2ll * F.nr);
    launch_uprow(F, C, prI, prW, prA, nullptr, st);
    int* fr = aalloc<int>(s->arena, 3ll * C.nr);
    double* frw = aalloc<double>(s->arena, 3ll * C.nr);
    int* longrows = aalloc<int>(s->arena, 2 * (C.nr + 1ll));
    launch_frows(F, C, prI, prW, prA, fr, frw, st);
    // staging for the sorted rows: a row has at most as many entries as
    // candidates, and a fine row feeds at most two coarse rows with two
    // columns per coupling, so 4 nnz of the fine level bound the total
    UStage ust;
    ust.toff = aalloc<int>(s->arena, C.nr);
    ust.cursor = aalloc<int>(s->arena, 1);
    ust.col = aalloc<int>(s->arena, 4 * F.nnz);
    ust.val = aalloc<double>(s->arena, 4 * F.nnz);
    ust.bits = aalloc<unsigned char>(s->arena, 4 * F.nnz);
    SSAMG_CUDA(cudaStreamWaitEvent(st, s->ev_uc, 0));
    launch_usort(F, C, longrows, fr, frw, C.u_ptr, ust, s->d_err, st);
    launch_scan(C.u_ptr, C.nr, scan_tmp, st);
    SSAMG_CUDA(cudaMemcpyAsync(s->h_int, C.u_ptr + C.nr, sizeof(int), cudaMemcpyDeviceToHost, st));
    SSAMG_CUDA(cudaStreamSynchronize(st));
    if (mark) SSAMG_CUDA(cudaEventSynchronize(s->ev_mark));
    C.nnz = s->h_int[0];
    C.u_col = aalloc<int>(s->arena, C.nnz);
    C.u_val = aalloc<double>(s->arena, C.nnz);
    C.u_bits = aalloc<unsigned char>(s->arena, C.nnz);
    if (fp32) C.u_val32 = aalloc<float>(s->arena, C.nnz);
    // the restriction onto C also pre-relaxes it (with U x): each coupling's
    // restriction row, made as the rows are copied
    C.u_rj = aalloc<int>(s->arena, 3 * C.nnz);
    C.u_rw = aalloc<double>(s->arena, 2 * C.nnz);
    if (fp32) C.u_rw32 = aalloc<float>(s->arena, 2 * C.nnz);
    launch_ucopy(F, C, ust, fp32, st);
    if (N2) {
      make_rows(*N2, s->h_int[1]);
      SSAMG_CUDA(cudaEventRecord(s->ev_rows, st));
    }
  }
  if (Lc > 0) SSAMG_CUDA(cudaStreamWaitEvent(st, s->ev_rap, 0));
  // has_u may be set on parts whose coarse rows vanished; refresh from U_c
  for (int l = 1; l <= Lc; ++l) {
    Level& L = s->lev[l];
    if (L.nr == 0) {
      bool changed = false;
      for (auto& h : L.parts)
        if (h.has_u) {
          h.has_u = 0;
          changed = true;
        }
      if (changed) upload_level(s, L, l < Lc ? &s->lev[l + 1] : nullptr, st);
    }
  }

  // ---- row-job data: dense U x buffers (one zeroed block); the P rows
  // (u_pj) and restriction rows (u_rj) of the coupling columns were made
  // with each level's P^T U P
  {
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    size_t total = 0;
    for (int l = 0; l <= Lc; ++l) {
      Level& L = s->lev[l];
      // lanes per row: the mean row length rounded up to a power of two,
      // between SSAMG_TPR and SSAMG_TPR_MAX (coarse levels' rows grow long)
      L.tpr = SSAMG_TPR;
      while (L.tpr < SSAMG_TPR_MAX && (long long)L.tpr * L.nr < L.nnz) L.tpr *= 2;
      L.nublk = (int)cdivll(L.nr, SSAMG_BLOCK / L.tpr);
      if (L.nr > 0) total += al(sizeof(double) * L.N) + (fp32 ? al(sizeof(float) * L.N) : 0);
    }
    if (total > 0) {
      char* base = (char*)s->arena.alloc(total);
      SSAMG_CUDA(cudaMemsetAsync(base, 0, total, st));
      for (int l = 0; l <= Lc; ++l) {
        Level& L = s->lev[l];
        if (L.nr == 0) continue;
        L.uy64 = (double*)base;
        base += al(sizeof(double) * L.N);
        if (fp32) {
          L.uy32 = (float*)base;
          base += al(sizeof(float) * L.N);
        }
      }
    }
  }

  // ---- Section 3.4: smoother diagonals
  // (level 0's were launched before the level loop) on the side stream,
  // beside the coarsest factor, which does not read them
  SSAMG_CUDA(cudaEventRecord(s->ev_p, st));
  SSAMG_CUDA(cudaStreamWaitEvent(s->ss, s->ev_p, 0));
  if (Lc > 0) launch_dinv(s->lev, 1, Lc, s->prm.relax, s->prm.relax_factor, fp32, s->ss);
  SSAMG_CUDA(cudaEventRecord(s->ev_rap, s->ss));

  // ---- coarsest level: dense Cholesky (FP64)
  Level& LL = s->lev[Lc];
  s->nL = (int)LL.N;
  if (s->prm.coarse_direct) {
    if (LL.N > 4096) throw SsamgError{SSAMG_ERR_UNSUPPORTED, "coarsest level too large for the dense solve"};
    s->chol = aalloc<double>(s->arena, LL.N * LL.N);
    launch_coarse_assemble(LL, s->chol, st);
    launch_cholesky((int)LL.N, s->chol, s->d_err + 2, st);
    if (LL.N <= 1024) {
      s->cinv = aalloc<double>(s->arena, LL.N * LL.N);
      launch_coarse_inverse((int)LL.N, s->chol, s->cinv, st);
    }
  }
  SSAMG_CUDA(cudaStreamWaitEvent(st, s->ev_rap, 0));
  // ---- fused coarse tail: the trailing levels that fit one block
  s->tail_lt = -1;
  s->tail_dev = nullptr;
  s->tail_bar = nullptr;
  if ((s->prm.use_tail == 1 || s->prm.use_tail == 2) && (!s->prm.coarse_direct || s->cinv)) {
    // use_tail 1: cooperative grid over the levels of at most
    // SSAMG_TAIL_MAX_CELLS cells; 2: one CTA over the levels of at most
    // tail_cells (default SSAMG_TAIL_CTA_CELLS) cells
    const bool one = s->prm.use_tail == 2;
    const long long maxc = one ? (s->prm.tail_cells > 0 ? s->prm.tail_cells : SSAMG_TAIL_CTA_CELLS)
                               : SSAMG_TAIL_MAX_CELLS;
    int lt = Lc;
    while (lt - 1 >= 0 && s->lev[lt - 1].N <= maxc && s->lev[lt - 1].np <= SSAMG_TAIL_MAX_PARTS)
      --lt;
    const int maxb = one ? 1 : tail_max_blocks();
    s->tail_parts = 0;
    for (int l = lt; l <= Lc; ++l) s->tail_parts += s->lev[l].np;
    bool fits = true;
    if (one && lt < Lc)
      fits = fp32 ? vtail_one_prepare<float>(Lc - lt + 1, s->tail_parts)
                  : vtail_one_prepare<double>(Lc - lt + 1, s->tail_parts);
    if (lt < Lc && fits && s->lev[lt].np <= SSAMG_TAIL_MAX_PARTS && maxb >= 1) {
      s->tail_lt = lt;
      s->tail_blocks = one ? 0
                           : (int)std::min<long long>(
                                 std::min<long long>(SSAMG_TAIL_MAX_BLOCKS, maxb),
                                 std::max<long long>(1, cdivll(s->lev[lt].N, SSAMG_TAIL_BLOCK)));
      if (!one) {
        s->tail_bar = aalloc<TailBarrier>(s->arena, 1);
        SSAMG_CUDA(cudaMemcpyAsync(s->tail_bar, &s->tail_bar_init, sizeof(TailBarrier),
                                   cudaMemcpyHostToDevice, st));
      }
      const int nt = Lc - lt + 1;
      if (fp32) {
        std::vector<TailLevel<float>> tl(nt);
        for (int l = lt; l <= Lc; ++l)
          tl[l - lt] = TailLevel<float>{s->lev[l].view<float>(), (float*)s->lev[l].x,
                                        (float*)s->lev[l].b, (float*)s->lev[l].r,
                                        (float*)s->lev[l].t, s->lev[l].shape, 0};
        s->tail_dev = s->arena.alloc(sizeof(TailLevel<float>) * nt);
        SSAMG_CUDA(cudaMemcpyAsync(s->tail_dev, tl.data(), sizeof(TailLevel<float>) * nt,
                                   cudaMemcpyHostToDevice, st));
      } else {
        std::vector<TailLevel<double>> tl(nt);
        for (int l = lt; l <= Lc; ++l)
          tl[l - lt] = TailLevel<double>{s->lev[l].view<double>(), (double*)s->lev[l].x,
                                         (double*)s->lev[l].b, (double*)s->lev[l].r,
                                         (double*)s->lev[l].t, s->lev[l].shape, 0};
        s->tail_dev = s->arena.alloc(sizeof(TailLevel<double>) * nt);
        SSAMG_CUDA(cudaMemcpyAsync(s->tail_dev, tl.data(), sizeof(TailLevel<double>) * nt,
                                   cudaMemcpyHostToDevice, st));
      }
    }
  }
  SSAMG_CUDA(cudaMemcpyAsync(s->h_int, s->d_err, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
  SSAMG_CUDA(cudaStreamSynchronize(st));
  if (s->h_int[0]) throw SsamgError{SSAMG_ERR_UNSUPPORTED, "a coarse coupling row has more than 1024 candidates"};
  if (s->h_int[2]) throw SsamgError{SSAMG_ERR_BREAKDOWN, "coarsest operator is not positive definite"};
  // ---- coarse-level transition in one cluster (use_tail = 3)
  s->ctail_lt = -1;
  if (s->prm.use_tail == 3) {
    NvtxRange nvt("ssamg setup transition");
    build_ctail(s, st);
  }

  // ---- PCG work vectors (the ones the level-0 stencil reads carry guard cells)
  long long N = s->lev[0].N;
  long long L0g = s->lev[0].guard;
  s->b = aalloc<double>(s->arena, N);
  s->x = (double*)padded_vector(s, sizeof(double), N, L0g, st);
  s->r = aalloc<double>(s->arena, N);
  s->z = aalloc<double>(s->arena, N);
  s->p = (double*)padded_vector(s, sizeof(double), N, L0g, st);
  s->q = aalloc<double>(s->arena, N);
  s->zprev = aalloc<double>(s->arena, N);
  s->partial = aalloc<double>(s->arena, 2ll * std::max(L0.nblk, L0.nbblk));
  s->tres = aalloc<double>(s->arena, 2ll * s->nprob);
  s->sc = aalloc<PcgScalars>(s->arena, s->nprob);
  s->ctl = aalloc<PcgCtl>(s->arena, 1);
  s->hist = aalloc<double>(s->arena, (long long)s->nprob * (s->prm.max_iter + 1));
  SSAMG_CUDA(cudaMemsetAsync(s->ctl, 0, sizeof(PcgCtl), st));
  {
    std::vector<PcgScalars> init(s->nprob);
    for (auto& v : init) {
      std::memset(&v, 0, sizeof(v));
      v.tol = s->prm.tol;
      v.max_iter = s->prm.max_iter;
      v.flexible = s->prm.flexible;
    }
    s->sc_init = aalloc<PcgScalars>(s->arena, s->nprob);
    SSAMG_CUDA(cudaMemcpyAsync(s->sc_init, init.data(), sizeof(PcgScalars) * s->nprob,
                               cudaMemcpyHostToDevice, st));
    SSAMG_CUDA(cudaStreamSynchronize(st));  // init is a host temporary
  }
  {
    // level-0 block and cell ranges of each problem (parts are problem-ordered)
    std::vector<int> hpb(s->nprob + 1, L0.nblk), hpbb(s->nprob + 1, L0.nbblk);
    s->prob_cells.assign(s->nprob + 1, N);
    for (int p = L0.np - 1; p >= 0; --p) {
      const int k = s->part_prob.empty() ? 0 : s->part_prob[p];
      hpb[k] = L0.hblk[p];
      hpbb[k] = L0.hbblk[p];
      s->prob_cells[k] = L0.parts[p].off;
    }
    s->pb = aalloc<int>(s->arena, s->nprob + 1);
    s->pbb = aalloc<int>(s->arena, s->nprob + 1);
    SSAMG_CUDA(cudaMemcpyAsync(s->pb, hpb.data(), sizeof(int) * (s->nprob + 1),
                               cudaMemcpyHostToDevice, st));
    SSAMG_CUDA(cudaMemcpyAsync(s->pbb, hpbb.data(), sizeof(int) * (s->nprob + 1),
                               cudaMemcpyHostToDevice, st));
    SSAMG_CUDA(cudaStreamSynchronize(st));  // hpb is a host temporary
  }
  s->ready = true;
}

// One V(1,1) cycle z = M r (r, z: FP64 level-0 vectors).
// One V(1,1) cycle z = M r.  With `dots` set, the last post-relaxation also
// produces the PCG's r.z (and r.zprev) block partials in `dots` and the
// function returns their block count (0: not fused, compute them apart).
template <class T>
int enqueue_vcycle(ssamg_solver s, const double* r_in, double* z_out, cudaStream_t st,
                   double* dots = nullptr, double* zprev = nullptr) {
  auto& Ls = s->lev;
  const int Lc = (int)Ls.size() - 1;
  const bool is_f = sizeof(T) == sizeof(float);
  const bool fused_in = is_f && Lc > 0 && s->tail_lt != 0;
  const T* b0;
  if (is_f) {
    if (!fused_in) launch_cast_d2f(r_in, (float*)Ls[0].b, Ls[0].N, st);
    b0 = (const T*)Ls[0].b;
  } else {
    b0 = (const T*)r_in;
  }
  auto coarse = [&](const T* bl, T* xl) {
    if (s->prm.coarse_direct && s->cinv)
      launch_coarse_apply<T>(s->nL, s->cinv, bl, xl, st);
    else if (s->prm.coarse_direct)
      launch_coarse_solve<T>(s->nL, s->chol, bl, xl, st);
    else
      launch_relax0<T>(Ls[Lc], bl, xl, st);
  };
  if (Lc == 0) {
    T* out = is_f ? (T*)Ls[0].t : (T*)z_out;
    coarse(b0, out);
    if (is_f) launch_cast_f2d((const float*)out, z_out, Ls[0].N, st);
    return 0;
  }
  // levels from tail_lt on run in one fused single-block launch, or from
  // ctail_lt on in one cluster
  const int lt = s->ctail_lt >= 1 ? s->ctail_lt : s->tail_lt >= 0 ? s->tail_lt : Lc;
  if (lt == 0) {
    // the whole cycle fits the tail: it reads b and writes t of level 0
    if (!is_f)
      SSAMG_CUDA(cudaMemcpyAsync(Ls[0].b, r_in, sizeof(double) * Ls[0].N, cudaMemcpyDeviceToDevice, st));
    launch_vtail<T>((const TailLevel<T>*)s->tail_dev, Lc + 1, s->cinv, s->nL, s->prm.coarse_direct,
                    s->tail_blocks, s->tail_bar, st, s->tail_parts);
    if (is_f)
      launch_cast_f2d((const float*)Ls[0].t, z_out, Ls[0].N, st);
    else
      SSAMG_CUDA(cudaMemcpyAsync(z_out, Ls[0].t, sizeof(double) * Ls[0].N, cudaMemcpyDeviceToDevice, st));
    return 0;
  }
  // down: pre-relax from zero (with U x for the residual), residual,
  // restrict; below level 0 the restriction also does the next level's
  // pre-relaxation (x = omega M^-1 b is pointwise; its row jobs rebuild b at
  // a coupling's column from the column's restriction row)
  const T* b = b0;
  for (int l = 0; l < lt; ++l) {
    T* x = (T*)Ls[l].x;
    T* r = (T*)Ls[l].r;
    if (l == 0 && fused_in)
      launch_relax0_u_first<T>(Ls[0], r_in, (T*)Ls[0].b, x, st);
    else if (l == 0)
      launch_relax0_u<T>(Ls[l], b, x, st);
    launch_residual<T>(Ls[l], x, b, r, st);
    launch_restrict<T>(Ls[l], Ls[l + 1], r, (T*)Ls[l + 1].b,
                       l + 1 < lt ? (T*)Ls[l + 1].x : nullptr, st);
    b = (const T*)Ls[l + 1].b;
  }
  const T* e;
  if (lt < Lc && s->ctail_lt == lt) {
    launch_ctail<T>(s->ctail, s->ctail_nc, s->ctail_smem, (const T*)Ls[lt].b, (T*)Ls[lt].t, st);
    e = (const T*)Ls[lt].t;
  } else if (lt < Lc) {
    launch_vtail<T>((const TailLevel<T>*)s->tail_dev, Lc - lt + 1, s->cinv, s->nL,
                    s->prm.coarse_direct, s->tail_blocks, s->tail_bar, st, s->tail_parts);
    e = (const T*)Ls[lt].t;
  } else {
    coarse((const T*)Ls[Lc].b, (T*)Ls[Lc].x);
    e = (const T*)Ls[Lc].x;
  }
  // up: x + P e into the (now free) residual buffer with U x, post-relax
  for (int l = lt - 1; l >= 0; --l) {
    T* xc = (T*)Ls[l].r;
    launch_prolong_u<T>(Ls[l], e, (const T*)Ls[l].x, xc, st);
    const T* bl = l == 0 ? b0 : (const T*)Ls[l].b;
    if (l == 0 && (dots || is_f)) {
      // straight into the FP64 z (and the PCG dot partials when asked)
      double* part = dots ? dots : s->partial;
      launch_relax_final<T>(Ls[0], xc, bl, z_out, r_in, dots ? zprev : nullptr, part, st);
      return dots ? Ls[0].nblk : 0;
    }
    T* out = (l == 0) ? (T*)z_out : (T*)Ls[l].t;
    launch_relax<T>(Ls[l], xc, bl, out, st);
    e = out;
  }
  return 0;
}

int vcycle(ssamg_solver s, const double* r, double* z, cudaStream_t st, double* dots = nullptr,
           double* zprev = nullptr) {
  if (s->prm.precision == 1) return enqueue_vcycle<float>(s, r, z, st, dots, zprev);
  return enqueue_vcycle<double>(s, r, z, st, dots, zprev);
}

// PCG segments.  init: r = b - A x; the first iteration is peeled so that the
// loop body starts with the V-cycle and ends with the convergence test.
PcgCtx pcg_ctx(ssamg_solver s) {
  return PcgCtx{s->pb, s->pbb, s->nprob, s->sc, s->ctl, s->partial, s->hist,
                s->prm.max_iter + 1, s->any_sc ? s->any_sc : s->sc,
                s->any_sc ? s->any_n : s->nprob};
}

void enqueue_pcg_head(ssamg_solver s, cudaGraphConditionalHandle h, int use_h, cudaStream_t st) {
  Level& L0 = s->lev[0];
  double* zp = s->prm.flexible ? s->zprev : nullptr;
  const PcgCtx c = pcg_ctx(s);
  SkipScope skip(s->sc);
  launch_pcg_init(L0, s->b, s->x, s->r, c, st);
  vcycle(s, s->r, s->z, st);
  launch_pcg_start(L0, s->r, s->z, s->p, zp, c, st);
  launch_pcg_alpha(L0, s->p, s->q, c, st);
  launch_pcg_update(L0, s->p, s->q, s->x, s->r, c, h, use_h, st);
}

void enqueue_pcg_body(ssamg_solver s, cudaGraphConditionalHandle h, int use_h, cudaStream_t st) {
  Level& L0 = s->lev[0];
  double* zp = s->prm.flexible ? s->zprev : nullptr;
  // the cycle's last kernel also forms r.z (and r.zprev) for beta
  const PcgCtx c = pcg_ctx(s);
  SkipScope skip(s->sc);
  const int npart = vcycle(s, s->r, s->z, st, s->partial, zp);
  if (npart > 0)  // the last relaxation writes partials per block of its tiles
    launch_pcg_beta_from_partials(L0, s->z, s->p, c, final_ranges(L0, c), st);
  else
    launch_pcg_beta(L0, s->r, s->z, zp, s->p, c, st);
  launch_pcg_alpha(L0, s->p, s->q, c, st);
  launch_pcg_update(L0, s->p, s->q, s->x, s->r, c, h, use_h, st);
}

void build_pcg_graph(ssamg_solver s) {
  if (!s->cs) SSAMG_CUDA(cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  SSAMG_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle h;
  SSAMG_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  // head, captured straight into g
  SSAMG_CUDA(cudaStreamBeginCaptureToGraph(s->cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  long long c0 = g_ssamg_launches;
  enqueue_pcg_head(s, h, 1, s->cs);
  s->head_launches = g_ssamg_launches - c0;
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  SSAMG_CUDA(cudaStreamGetCaptureInfo(s->cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps));
  std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
  cudaGraph_t tmp;
  SSAMG_CUDA(cudaStreamEndCapture(s->cs, &tmp));
  // while node: body = one PCG iteration
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  SSAMG_CUDA(cudaGraphAddNode(&cnode, g, tail.data(), nullptr, tail.size(), &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  SSAMG_CUDA(cudaStreamBeginCaptureToGraph(s->cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  c0 = g_ssamg_launches;
  enqueue_pcg_body(s, h, 1, s->cs);
  s->body_launches = g_ssamg_launches - c0;
  SSAMG_CUDA(cudaStreamEndCapture(s->cs, &tmp));
  SSAMG_CUDA(cudaGraphInstantiate(&s->graphs.pcg, g, 0));
  cudaGraphDestroy(g);
}

// Per-problem statistics from host copies of the PCG scalars and of the
// (||b||^2, ||b - A x||^2) pairs.
void fill_stats(ssamg_solver s, ssamg_stats* stats, const PcgScalars* sc, const double* tres) {
  const int np = s->nprob;
  int maxit = 0;
  for (int k = 0; k < np; ++k) maxit = std::max(maxit, sc[k].iter);
  double nnz0 = 0, nnz = 0;
  for (size_t l = 0; l < s->lev.size(); ++l) {
    double n = (double)s->lev[l].nnz;
    for (auto& h : s->lev[l].parts) n += (double)h.nent * h.ncell;
    nnz += n;
    if (l == 0) nnz0 = n;
  }
  for (int k = 0; k < np; ++k) {
    const PcgScalars& r = sc[k];
    ssamg_stats& o = stats[k];
    o.iterations = r.iter;
    o.setup_kernel_launches = s->setup_launches;
    // the loop runs until the slowest problem stops
    o.solve_kernel_launches = s->head_launches + (long long)(maxit > 0 ? maxit - 1 : 0) * s->body_launches;
    o.converged = r.status == 0 && r.rr <= r.tol2bb;
    o.rel_res = r.bb > 0 ? std::sqrt(r.rr / r.bb) : 0.0;
    o.num_levels = (int)s->lev.size();
    o.coarse_size = s->lev.back().N;
    o.operator_complexity = nnz / nnz0;
    o.true_rel_res = tres[2 * k] > 0 ? std::sqrt(tres[2 * k + 1] / tres[2 * k]) : 0.0;
  }
}

int worst_status(ssamg_solver s, const PcgScalars* sc) {
  int rc = SSAMG_OK;
  for (int k = 0; k < s->nprob; ++k) {
    if (sc[k].status != 0) return sc[k].status;
    if (!(sc[k].rr <= sc[k].tol2bb)) rc = SSAMG_NOT_CONVERGED;
  }
  return rc;
}

// One graph for `nrhs` solves in a row (right-hand side j at b + j N, its
// solution to x + j N): per round, the right-hand side is copied in, x and
// the scalars reset, the PCG head and its while loop run, and the solution,
// the scalars and the true-residual sums are copied out to the history.
void build_rounds_graph(ssamg_solver s, const double* b, double* x, int nrhs, int zero_guess) {
  if (!s->cs) SSAMG_CUDA(cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking));
  const long long N = s->lev[0].N;
  const int np = s->nprob;
  cudaGraph_t g;
  SSAMG_CUDA(cudaGraphCreate(&g, 0));
  std::vector<cudaGraphNode_t> deps;
  cudaStreamCaptureStatus cst;
  const cudaGraphNode_t* dp = nullptr;
  size_t ndp = 0;
  cudaGraph_t tmp;
  auto begin = [&](cudaGraph_t gg, const std::vector<cudaGraphNode_t>& d) {
    SSAMG_CUDA(cudaStreamBeginCaptureToGraph(s->cs, gg, d.empty() ? nullptr : d.data(), nullptr,
                                             d.size(), cudaStreamCaptureModeThreadLocal));
  };
  auto end = [&]() {
    SSAMG_CUDA(cudaStreamGetCaptureInfo(s->cs, &cst, nullptr, nullptr, &dp, nullptr, &ndp));
    std::vector<cudaGraphNode_t> t(dp, dp + ndp);
    SSAMG_CUDA(cudaStreamEndCapture(s->cs, &tmp));
    return t;
  };
  for (int j = 0; j < nrhs; ++j) {
    cudaGraphConditionalHandle h;
    SSAMG_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    begin(g, deps);
    SSAMG_CUDA(cudaMemcpyAsync(s->b, b + j * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, s->cs));
    if (zero_guess)
      SSAMG_CUDA(cudaMemsetAsync(s->x, 0, sizeof(double) * N, s->cs));
    else
      SSAMG_CUDA(cudaMemcpyAsync(s->x, x + j * N, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                                 s->cs));
    SSAMG_CUDA(cudaMemcpyAsync(s->sc, s->sc_init, sizeof(PcgScalars) * np, cudaMemcpyDeviceToDevice,
                               s->cs));
    long long c0 = g_ssamg_launches;
    enqueue_pcg_head(s, h, 1, s->cs);
    s->head_launches = g_ssamg_launches - c0;
    std::vector<cudaGraphNode_t> tail = end();
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    SSAMG_CUDA(cudaGraphAddNode(&cnode, g, tail.data(), nullptr, tail.size(), &cp));
    begin(cp.conditional.phGraph_out[0], {});
    c0 = g_ssamg_launches;
    enqueue_pcg_body(s, h, 1, s->cs);
    s->body_launches = g_ssamg_launches - c0;
    end();
    begin(g, {cnode});
    SSAMG_CUDA(cudaMemcpyAsync(x + j * N, s->x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s->cs));
    launch_true_residual(s->lev[0], s->b, s->x, s->q, pcg_ctx(s), s->tres_hist + 2ll * j * np,
                         s->cs);
    SSAMG_CUDA(cudaMemcpyAsync(s->sc_hist + (long long)j * np, s->sc, sizeof(PcgScalars) * np,
                               cudaMemcpyDeviceToDevice, s->cs));
    deps = end();
  }
  if (s->graphs.rounds) cudaGraphExecDestroy(s->graphs.rounds);
  s->graphs.rounds = nullptr;
  SSAMG_CUDA(cudaGraphInstantiate(&s->graphs.rounds, g, 0));
  cudaGraphDestroy(g);
  s->graphs.rounds_b = b;
  s->graphs.rounds_x = x;
  s->graphs.rounds_n = nrhs;
  s->graphs.rounds_zero = zero_guess;
}

// ---- Right-hand sides solved together --------------------------------------
// One PCG loop runs every right-hand side of a batch: each step of the cycle
// is enqueued for right-hand side 0, 1, ... in turn (its vectors swapped into
// the solver), except the residual and the relaxation on cell-tile levels,
// which take all right-hand sides in one launch with the blocks of a tile
// side by side, so that the tile's stencil coefficients come from HBM once
// and from L2 for the others.  Every right-hand side computes what it would
// alone, in the same order.

// First level of the coarse tail the host-side cycle stops at (as in
// enqueue_vcycle).
int cycle_tail_level(ssamg_solver s) {
  const int Lc = (int)s->lev.size() - 1;
  return s->ctail_lt >= 1 ? s->ctail_lt : s->tail_lt >= 0 ? s->tail_lt : Lc;
}

// Whether the right-hand sides can share launches: a cycle with levels above
// its tail and no fused grid-barrier tail (whose level table holds one set of
// vectors).
bool rhs_together_ok(ssamg_solver s) {
  const int Lc = (int)s->lev.size() - 1;
  return Lc > 0 && s->tail_lt < 0 && cycle_tail_level(s) > 0;
}

struct RhsSaved {
  double *b, *x, *r, *z, *p, *q, *zprev, *partial, *hist;
  PcgScalars* sc;
  std::vector<void*> x_, b_, r_, t_;
  std::vector<float*> uy32;
  std::vector<double*> uy64;
};

// Slices for R right-hand sides (kept until the next set-up, and reused by
// solves of as many right-hand sides or fewer); zeroed on st.
void alloc_rhs(ssamg_solver s, int R, cudaStream_t st) {
  RhsSet& M = s->rhs;
  if (M.cap >= R) {
    M.R = R;
    return;
  }
  const bool fp32 = s->prm.precision == 1;
  const size_t w = fp32 ? sizeof(float) : sizeof(double);
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  auto slab = [](long long n, long long guard) { return (n + 2 * guard + 63) / 64 * 64; };
  RhsSet N;
  N.R = N.cap = R;
  N.nlev = cycle_tail_level(s) + 1;
  N.stride.resize(N.nlev);
  size_t total = 0;
  for (int l = 0; l < N.nlev; ++l) {
    const Level& L = s->lev[l];
    N.stride[l] = slab(L.N, L.guard);
    total += 4 * al(w * N.stride[l] * R);
    if (L.nr > 0) total += al(8 * N.stride[l] * R) + (fp32 ? al(4 * N.stride[l] * R) : 0);
  }
  const Level& L0 = s->lev[0];
  N.stride0 = slab(L0.N, L0.guard);  // equal to stride[0] (element counts)
  total += 7 * al(8 * N.stride0 * R);
  N.partial_len = 2ll * std::max(L0.nblk, L0.nbblk);
  total += al(8 * N.partial_len * R);
  total += al(sizeof(PcgScalars) * (size_t)s->nprob * R);
  N.hist_len = (long long)s->nprob * (s->prm.max_iter + 1);
  total += al(8 * N.hist_len * R);
  char* base = (char*)s->arena.alloc(total);
  SSAMG_CUDA(cudaMemsetAsync(base, 0, total, st));
  auto take = [&](size_t bytes) {
    char* p = base;
    base += al(bytes);
    return p;
  };
  N.x.resize(N.nlev);
  N.b.resize(N.nlev);
  N.r.resize(N.nlev);
  N.t.resize(N.nlev);
  N.uy32.assign(N.nlev, nullptr);
  N.uy64.assign(N.nlev, nullptr);
  for (int l = 0; l < N.nlev; ++l) {
    const Level& L = s->lev[l];
    const size_t g = w * L.guard;
    N.x[l] = take(w * N.stride[l] * R) + g;
    N.b[l] = take(w * N.stride[l] * R) + g;
    N.r[l] = take(w * N.stride[l] * R) + g;
    N.t[l] = take(w * N.stride[l] * R) + g;
    if (L.nr > 0) {
      N.uy64[l] = (double*)take(8 * N.stride[l] * R);
      if (fp32) N.uy32[l] = (float*)take(4 * N.stride[l] * R);
    }
  }
  double** pv[7] = {&N.pb, &N.px, &N.pr, &N.pz, &N.pp, &N.pq, &N.pzprev};
  for (double** q : pv) *q = (double*)take(8 * N.stride0 * R) + L0.guard;
  N.partial = (double*)take(8 * N.partial_len * R);
  N.sc = (PcgScalars*)take(sizeof(PcgScalars) * (size_t)s->nprob * R);
  N.hist = (double*)take(8 * N.hist_len * R);
  M = std::move(N);
}

RhsSaved save_rhs(ssamg_solver s) {
  RhsSaved o{s->b, s->x, s->r, s->z, s->p, s->q, s->zprev, s->partial, s->hist, s->sc,
             {}, {}, {}, {}, {}, {}};
  for (int l = 0; l < s->rhs.nlev; ++l) {
    const Level& L = s->lev[l];
    o.x_.push_back(L.x);
    o.b_.push_back(L.b);
    o.r_.push_back(L.r);
    o.t_.push_back(L.t);
    o.uy32.push_back(L.uy32);
    o.uy64.push_back(L.uy64);
  }
  return o;
}

void restore_rhs(ssamg_solver s, const RhsSaved& o) {
  s->b = o.b;
  s->x = o.x;
  s->r = o.r;
  s->z = o.z;
  s->p = o.p;
  s->q = o.q;
  s->zprev = o.zprev;
  s->partial = o.partial;
  s->hist = o.hist;
  s->sc = o.sc;
  for (int l = 0; l < s->rhs.nlev; ++l) {
    Level& L = s->lev[l];
    L.x = o.x_[l];
    L.b = o.b_[l];
    L.r = o.r_[l];
    L.t = o.t_[l];
    L.uy32 = o.uy32[l];
    L.uy64 = o.uy64[l];
  }
}

// Right-hand side j's slices into the solver (and its scalars into the
// level views' skip pointer).
void use_rhs(ssamg_solver s, int j) {
  const RhsSet& M = s->rhs;
  const bool fp32 = s->prm.precision == 1;
  const size_t w = fp32 ? sizeof(float) : sizeof(double);
  const long long o0 = j * M.stride0;
  s->b = M.pb + o0;
  s->x = M.px + o0;
  s->r = M.pr + o0;
  s->z = M.pz + o0;
  s->p = M.pp + o0;
  s->q = M.pq + o0;
  s->zprev = M.pzprev + o0;
  s->partial = M.partial + j * M.partial_len;
  s->hist = M.hist + j * M.hist_len;
  s->sc = M.sc + (long long)j * s->nprob;
  for (int l = 0; l < M.nlev; ++l) {
    Level& L = s->lev[l];
    const long long o = j * M.stride[l];
    L.x = M.x[l] + w * o;
    L.b = M.b[l] + w * o;
    L.r = M.r[l] + w * o;
    L.t = M.t[l] + w * o;
    L.uy32 = M.uy32[l] ? M.uy32[l] + o : nullptr;
    L.uy64 = M.uy64[l] ? M.uy64[l] + o : nullptr;
  }
  g_ssamg_skip = s->sc;
}

// The V(1,1) cycle z_j = M r_j of every right-hand side j (r, z: the PCG
// slices).  With `dots`, the last relaxation also forms each right-hand
// side's r.z (and r.zprev) partials in its own buffer; returns their block
// count as enqueue_vcycle does.
template <class T>
int enqueue_vcycle_rhs(ssamg_solver s, bool dots, cudaStream_t st) {
  const RhsSet& M = s->rhs;
  const int R = M.R;
  auto& Ls = s->lev;
  const int Lc = (int)Ls.size() - 1;
  const bool is_f = sizeof(T) == sizeof(float);
  const bool fused_in = is_f && s->tail_lt != 0;
  const int lt = cycle_tail_level(s);
  const bool ctail = lt < Lc && s->ctail_lt == lt;
  auto each = [&](auto&& f) {
    for (int j = 0; j < R; ++j) {
      use_rhs(s, j);
      f();
    }
    use_rhs(s, 0);
  };
  // right-hand side's level-0 cycle right-hand side (slice of the current one)
  auto b0 = [&]() { return is_f ? (const T*)Ls[0].b : (const T*)s->r; };
  auto coarse = [&](const T* bl, T* xl) {
    if (s->prm.coarse_direct && s->cinv)
      launch_coarse_apply<T>(s->nL, s->cinv, bl, xl, st);
    else if (s->prm.coarse_direct)
      launch_coarse_solve<T>(s->nL, s->chol, bl, xl, st);
    else
      launch_relax0<T>(Ls[Lc], bl, xl, st);
  };
  for (int l = 0; l < lt; ++l) {
    if (l == 0)
      each([&] {
        if (fused_in) {
          launch_relax0_u_first<T>(Ls[0], s->r, (T*)Ls[0].b, (T*)Ls[0].x, st);
        } else {
          if (is_f) launch_cast_d2f(s->r, (float*)Ls[0].b, Ls[0].N, st);
          launch_relax0_u<T>(Ls[0], b0(), (T*)Ls[0].x, st);
        }
      });
    if (!uses_bricks(Ls[l])) {
      use_rhs(s, 0);
      launch_residual_rhs<T>(Ls[l], R, M.stride[l], s->nprob, (const T*)Ls[l].x,
                             l == 0 ? b0() : (const T*)Ls[l].b, (T*)Ls[l].r, st);
    } else {
      each([&] {
        launch_residual<T>(Ls[l], (const T*)Ls[l].x, l == 0 ? b0() : (const T*)Ls[l].b,
                           (T*)Ls[l].r, st);
      });
    }
    each([&] {
      launch_restrict<T>(Ls[l], Ls[l + 1], (const T*)Ls[l].r, (T*)Ls[l + 1].b,
                         l + 1 < lt ? (T*)Ls[l + 1].x : nullptr, st);
    });
  }
  each([&] {
    if (ctail)
      launch_ctail<T>(s->ctail, s->ctail_nc, s->ctail_smem, (const T*)Ls[lt].b, (T*)Ls[lt].t, st);
    else
      coarse((const T*)Ls[Lc].b, (T*)Ls[Lc].x);
  });
  // the correction prolongated to level l comes from level l + 1's output
  auto e_of = [&](int l) {
    if (l + 1 == lt) return ctail ? (const T*)Ls[lt].t : (const T*)Ls[Lc].x;
    return (const T*)Ls[l + 1].t;
  };
  for (int l = lt - 1; l >= 0; --l) {
    each([&] { launch_prolong_u<T>(Ls[l], e_of(l), (const T*)Ls[l].x, (T*)Ls[l].r, st); });
    if (l == 0 && (dots || is_f)) {
      each([&] {
        launch_relax_final<T>(Ls[0], (const T*)Ls[0].r, b0(), s->z, s->r,
                              dots ? s->zprev : nullptr, s->partial, st);
      });
      return dots ? Ls[0].nblk : 0;
    }
    if (!uses_bricks(Ls[l])) {
      use_rhs(s, 0);
      T* out = l == 0 ? (T*)s->z : (T*)Ls[l].t;
      launch_relax_rhs<T>(Ls[l], R, M.stride[l], s->nprob, (const T*)Ls[l].r,
                          l == 0 ? b0() : (const T*)Ls[l].b, out, st);
    } else {
      each([&] {
        T* out = l == 0 ? (T*)s->z : (T*)Ls[l].t;
        launch_relax<T>(Ls[l], (const T*)Ls[l].r, l == 0 ? b0() : (const T*)Ls[l].b, out, st);
      });
    }
  }
  return 0;
}

int vcycle_rhs(ssamg_solver s, bool dots, cudaStream_t st) {
  if (s->prm.precision == 1) return enqueue_vcycle_rhs<float>(s, dots, st);
  return enqueue_vcycle_rhs<double>(s, dots, st);
}

// PCG head and loop body of every right-hand side (as enqueue_pcg_head /
// enqueue_pcg_body; the scalar steps per right-hand side, the cycle shared).
void enqueue_pcg_head_rhs(ssamg_solver s, cudaGraphConditionalHandle h, cudaStream_t st) {
  const int R = s->rhs.R;
  Level& L0 = s->lev[0];
  for (int j = 0; j < R; ++j) {
    use_rhs(s, j);
    launch_pcg_init(L0, s->b, s->x, s->r, pcg_ctx(s), st);
  }
  vcycle_rhs(s, false, st);
  for (int j = 0; j < R; ++j) {
    use_rhs(s, j);
    const PcgCtx c = pcg_ctx(s);
    launch_pcg_start(L0, s->r, s->z, s->p, s->prm.flexible ? s->zprev : nullptr, c, st);
    launch_pcg_alpha(L0, s->p, s->q, c, st);
    launch_pcg_update(L0, s->p, s->q, s->x, s->r, c, h, 1, st);
  }
}

void enqueue_pcg_body_rhs(ssamg_solver s, cudaGraphConditionalHandle h, cudaStream_t st) {
  const int R = s->rhs.R;
  Level& L0 = s->lev[0];
  const int npart = vcycle_rhs(s, true, st);
  for (int j = 0; j < R; ++j) {
    use_rhs(s, j);
    const PcgCtx c = pcg_ctx(s);
    double* zp = s->prm.flexible ? s->zprev : nullptr;
    if (npart > 0)
      launch_pcg_beta_from_partials(L0, s->z, s->p, c, final_ranges(L0, c), st);
    else
      launch_pcg_beta(L0, s->r, s->z, zp, s->p, c, st);
    launch_pcg_alpha(L0, s->p, s->q, c, st);
    launch_pcg_update(L0, s->p, s->q, s->x, s->r, c, h, 1, st);
  }
}

// One graph for nrhs right-hand sides solved together (right-hand side j at
// b + j N, its solution to x + j N): the right-hand sides are copied in and
// x and the scalars reset, the shared PCG head and while loop run, and the
// solutions, scalars and true-residual sums are copied out to the history
// (the last right-hand side's residual history and scalars to the solver's).
void build_rhs_graph(ssamg_solver s, const double* b, double* x, int nrhs, int zero_guess) {
  if (!s->cs) SSAMG_CUDA(cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking));
  const long long N = s->lev[0].N;
  const int np = s->nprob;
  const RhsSaved saved = save_rhs(s);
  SkipScope skip(s->rhs.sc);
  s->any_sc = s->rhs.sc;
  s->any_n = nrhs * np;
  cudaGraph_t g = nullptr;
  try {
    SSAMG_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    SSAMG_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t* dp = nullptr;
    size_t ndp = 0;
    cudaGraph_t tmp;
    SSAMG_CUDA(cudaStreamBeginCaptureToGraph(s->cs, g, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
    for (int j = 0; j < nrhs; ++j) {
      use_rhs(s, j);
      SSAMG_CUDA(cudaMemcpyAsync(s->b, b + j * N, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                                 s->cs));
      if (zero_guess)
        SSAMG_CUDA(cudaMemsetAsync(s->x, 0, sizeof(double) * N, s->cs));
      else
        SSAMG_CUDA(cudaMemcpyAsync(s->x, x + j * N, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                                   s->cs));
      SSAMG_CUDA(cudaMemcpyAsync(s->sc, s->sc_init, sizeof(PcgScalars) * np,
                                 cudaMemcpyDeviceToDevice, s->cs));
    }
    long long c0 = g_ssamg_launches;
    enqueue_pcg_head_rhs(s, h, s->cs);
    s->head_launches = g_ssamg_launches - c0;
    SSAMG_CUDA(cudaStreamGetCaptureInfo(s->cs, &cst, nullptr, nullptr, &dp, nullptr, &ndp));
    std::vector<cudaGraphNode_t> tail(dp, dp + ndp);
    SSAMG_CUDA(cudaStreamEndCapture(s->cs, &tmp));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    SSAMG_CUDA(cudaGraphAddNode(&cnode, g, tail.data(), nullptr, tail.size(), &cp));
    SSAMG_CUDA(cudaStreamBeginCaptureToGraph(s->cs, cp.conditional.phGraph_out[0], nullptr,
                                             nullptr, 0, cudaStreamCaptureModeThreadLocal));
    c0 = g_ssamg_launches;
    enqueue_pcg_body_rhs(s, h, s->cs);
    s->body_launches = g_ssamg_launches - c0;
    SSAMG_CUDA(cudaStreamEndCapture(s->cs, &tmp));
    SSAMG_CUDA(cudaStreamBeginCaptureToGraph(s->cs, g, &cnode, nullptr, 1,
                                             cudaStreamCaptureModeThreadLocal));
    for (int j = 0; j < nrhs; ++j) {
      use_rhs(s, j);
      SSAMG_CUDA(cudaMemcpyAsync(x + j * N, s->x, sizeof(double) * N, cudaMemcpyDeviceToDevice,
                                 s->cs));
      launch_true_residual(s->lev[0], s->b, s->x, s->q, pcg_ctx(s), s->tres_hist + 2ll * j * np,
                           s->cs);
      SSAMG_CUDA(cudaMemcpyAsync(s->sc_hist + (long long)j * np, s->sc, sizeof(PcgScalars) * np,
                                 cudaMemcpyDeviceToDevice, s->cs));
    }
    SSAMG_CUDA(cudaMemcpyAsync(saved.hist, s->hist, sizeof(double) * s->rhs.hist_len,
                               cudaMemcpyDeviceToDevice, s->cs));
    SSAMG_CUDA(cudaMemcpyAsync(saved.sc, s->sc, sizeof(PcgScalars) * np,
                               cudaMemcpyDeviceToDevice, s->cs));
    SSAMG_CUDA(cudaStreamEndCapture(s->cs, &tmp));
    if (s->graphs.rounds) cudaGraphExecDestroy(s->graphs.rounds);
    s->graphs.rounds = nullptr;
    SSAMG_CUDA(cudaGraphInstantiate(&s->graphs.rounds, g, 0));
  } catch (...) {
    // leave the capture stream usable: end a capture the error interrupted
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s->cs, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
      cudaGraph_t part = nullptr;
      cudaStreamEndCapture(s->cs, &part);
      if (part) cudaGraphDestroy(part);
    }
    restore_rhs(s, saved);
    s->any_sc = nullptr;
    if (g) cudaGraphDestroy(g);
    throw;
  }
  restore_rhs(s, saved);
  s->any_sc = nullptr;
  cudaGraphDestroy(g);
  s->graphs.rounds_b = b;
  s->graphs.rounds_x = x;
  s->graphs.rounds_n = nrhs;
  s->graphs.rounds_zero = zero_guess;
}

// Solves for nrhs right-hand sides (b, x: nrhs x N, device) in one graph
// launch; stats (nrhs x nprob) as for run_pcg.  One synchronisation.
int run_rounds(ssamg_solver s, const double* b, double* x, int nrhs, cudaStream_t st,
               ssamg_stats* stats, int zero_guess = 1) {
  const int np = s->nprob;
  if (s->hist_cap < nrhs) {
    if (s->sc_hist) cudaFree(s->sc_hist);
    if (s->tres_hist) cudaFree(s->tres_hist);
    s->sc_hist = nullptr;
    s->tres_hist = nullptr;
    s->hist_cap = 0;
    SSAMG_CUDA(cudaMalloc(&s->sc_hist, sizeof(PcgScalars) * np * nrhs));
    SSAMG_CUDA(cudaMalloc(&s->tres_hist, sizeof(double) * 2 * np * nrhs));
    s->hist_cap = nrhs;
    if (s->graphs.rounds) cudaGraphExecDestroy(s->graphs.rounds);
    s->graphs.rounds = nullptr;
  }
  if (!s->graphs.rounds || s->graphs.rounds_b != b || s->graphs.rounds_x != x ||
      s->graphs.rounds_n != nrhs || s->graphs.rounds_zero != zero_guess) {
    if (nrhs > 1 && s->prm.rhs_together && rhs_together_ok(s)) {
      alloc_rhs(s, nrhs, st);
      build_rhs_graph(s, b, x, nrhs, zero_guess);
    } else {
      build_rounds_graph(s, b, x, nrhs, zero_guess);
    }
  }
  SSAMG_CUDA(cudaGraphLaunch(s->graphs.rounds, st));
  std::vector<PcgScalars> sc((size_t)np * nrhs);
  std::vector<double> tres((size_t)2 * np * nrhs);
  SSAMG_CUDA(cudaMemcpyAsync(sc.data(), s->sc_hist, sizeof(PcgScalars) * np * nrhs,
                             cudaMemcpyDeviceToHost, st));
  SSAMG_CUDA(cudaMemcpyAsync(tres.data(), s->tres_hist, sizeof(double) * 2 * np * nrhs,
                             cudaMemcpyDeviceToHost, st));
  SSAMG_CUDA(cudaStreamSynchronize(st));
  if (s->tail_bar) {
    SSAMG_CUDA(cudaMemcpyAsync(s->h_int, &s->tail_bar->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SSAMG_CUDA(cudaStreamSynchronize(st));
    if (s->h_int[0]) {
      SSAMG_CUDA(cudaMemsetAsync(&s->tail_bar->err, 0, sizeof(int), st));
      throw SsamgError{SSAMG_ERR_TIMEOUT, "a grid barrier of the coarse-level kernel timed out"};
    }
  }
  int rc = SSAMG_OK;
  for (int j = 0; j < nrhs; ++j) {
    if (stats) fill_stats(s, stats + (long long)j * np, sc.data() + (long long)j * np,
                          tres.data() + 2ll * j * np);
    const int r = worst_status(s, sc.data() + (long long)j * np);
    if (r < 0) return r;
    if (r > rc) rc = r;
  }
  return rc;
}


// Runs the PCG of every problem of the solver on s->b, s->x (x0 given);
// stats, when set, receives one entry per problem.  Returns the worst status.
int run_pcg(ssamg_solver s, cudaStream_t st, ssamg_stats* stats) {
  const int np = s->nprob;
  SSAMG_CUDA(cudaMemcpyAsync(s->sc, s->sc_init, sizeof(PcgScalars) * np, cudaMemcpyDeviceToDevice, st));
  if (s->prm.use_graph) {
    if (!s->graphs.pcg) build_pcg_graph(s);
    SSAMG_CUDA(cudaGraphLaunch(s->graphs.pcg, st));
  } else {
    long long c0 = g_ssamg_launches;
    enqueue_pcg_head(s, 0, 0, st);
    s->head_launches = g_ssamg_launches - c0;
    for (;;) {
      SSAMG_CUDA(cudaMemcpyAsync(s->h_int, &s->ctl->active, sizeof(int), cudaMemcpyDeviceToHost, st));
      SSAMG_CUDA(cudaStreamSynchronize(st));
      if (!s->h_int[0]) break;
      c0 = g_ssamg_launches;
      enqueue_pcg_body(s, 0, 0, st);
      s->body_launches = g_ssamg_launches - c0;
    }
  }
  SSAMG_CUDA(cudaMemcpyAsync(s->h_sc, s->sc, sizeof(PcgScalars) * np, cudaMemcpyDeviceToHost, st));
  SSAMG_CUDA(cudaStreamSynchronize(st));
  if (s->tail_bar) {
    SSAMG_CUDA(cudaMemcpyAsync(s->h_int, &s->tail_bar->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SSAMG_CUDA(cudaStreamSynchronize(st));
    if (s->h_int[0]) {
      SSAMG_CUDA(cudaMemsetAsync(&s->tail_bar->err, 0, sizeof(int), st));
      throw SsamgError{SSAMG_ERR_TIMEOUT, "a grid barrier of the coarse-level kernel timed out"};
    }
  }
  if (stats) {
    launch_true_residual(s->lev[0], s->b, s->x, s->q, pcg_ctx(s), s->tres, st);
    SSAMG_CUDA(cudaMemcpyAsync(s->h_dbl, s->tres, sizeof(double) * 2 * np, cudaMemcpyDeviceToHost, st));
    SSAMG_CUDA(cudaStreamSynchronize(st));
    fill_stats(s, stats, s->h_sc, s->h_dbl);
  }
  return worst_status(s, s->h_sc);
}

}  // namespace

void run_setup(ssamg_solver s, cudaStream_t st) {
  noalloc_scratch();
  const long long c0 = g_ssamg_launches;
  build_hierarchy(s, st);
  s->setup_launches = g_ssamg_launches - c0;
}

extern "C" int ssamg_setup(ssamg_solver s, ssamg_matrix A, void* stream) {
  NvtxRange nv("ssamg_setup");
  if (!s || !A) return SSAMG_ERR_ARG;
  if (!A->assembled) return SSAMG_ERR_STATE;
  API_BEGIN
  s->A = A;
  run_setup(s, (cudaStream_t)stream);
  return SSAMG_OK;
  API_END
}

extern "C" int ssamg_solve(ssamg_solver s, const double* b, double* x, int nrhs, int zero_guess,
                           void* stream, ssamg_stats* st) {
  NvtxRange nv("ssamg_solve");
  if (!s || !b || !x || nrhs < 1) return SSAMG_ERR_ARG;
  if (!s->ready) return SSAMG_ERR_STATE;
  cudaStream_t cst = (cudaStream_t)stream;
  API_BEGIN
  PdlScope pdl(s->prm);
  if (nrhs > 1 && s->prm.use_graph) {
    // every right-hand side in one graph launch; st: the last one's stats
    std::vector<ssamg_stats> all(st ? (size_t)nrhs * s->nprob : 0);
    const int r = run_rounds(s, b, x, nrhs, cst, st ? all.data() : nullptr, zero_guess ? 1 : 0);
    if (st) std::copy(all.end() - s->nprob, all.end(), st);
    return r;
  }
  long long N = s->lev[0].N;
  int rc = SSAMG_OK;
  for (int k = 0; k < nrhs; ++k) {
    SSAMG_CUDA(cudaMemcpyAsync(s->b, b + k * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, cst));
    if (zero_guess)
      SSAMG_CUDA(cudaMemsetAsync(s->x, 0, sizeof(double) * N, cst));
    else
      SSAMG_CUDA(cudaMemcpyAsync(s->x, x + k * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, cst));
    int r = run_pcg(s, cst, st);
    SSAMG_CUDA(cudaMemcpyAsync(x + k * N, s->x, sizeof(double) * N, cudaMemcpyDeviceToDevice, cst));
    if (r < 0) return r;
    if (r > rc) rc = r;
  }
  return rc;
  API_END
}

extern "C" int ssamg_solve_host(ssamg_solver s, const double* b, double* x, int nrhs, void* stream,
                                ssamg_stats* st) {
  if (!s || !b || !x || nrhs < 1) return SSAMG_ERR_ARG;
  if (!s->ready) return SSAMG_ERR_STATE;
  cudaStream_t cst = (cudaStream_t)stream;
  API_BEGIN
  PdlScope pdl(s->prm);
  long long N = s->lev[0].N;
  int rc = SSAMG_OK;
  for (int k = 0; k < nrhs; ++k) {
    SSAMG_CUDA(cudaMemcpyAsync(s->b, b + k * N, sizeof(double) * N, cudaMemcpyHostToDevice, cst));
    SSAMG_CUDA(cudaMemsetAsync(s->x, 0, sizeof(double) * N, cst));
    int r = run_pcg(s, cst, st);
    SSAMG_CUDA(cudaMemcpyAsync(x + k * N, s->x, sizeof(double) * N, cudaMemcpyDeviceToHost, cst));
    SSAMG_CUDA(cudaStreamSynchronize(cst));
    if (r < 0) return r;
    if (r > rc) rc = r;
  }
  return rc;
  API_END
}

extern "C" int ssamg_adjoint_solve(ssamg_solver s, const double* g, double* lambda, int nrhs,
                                   void* stream, ssamg_stats* st) {
  // A is symmetric (S by the caller's stencil, U by assumption), so the
  // adjoint system A^T lambda = g is solved with the forward hierarchy.
  return ssamg_solve(s, g, lambda, nrhs, 1, stream, st);
}

extern "C" int ssamg_coef_gradient(ssamg_solver s, const double* lambda, const double* x,
                                   double* dcoef, void* stream) {
  if (!s || !lambda || !x || !dcoef) return SSAMG_ERR_ARG;
  if (!s->ready) return SSAMG_ERR_STATE;
  API_BEGIN
  PdlScope pdl(s->prm);
  launch_coef_gradient(s->lev[0], lambda, x, dcoef, (cudaStream_t)stream);
  return SSAMG_OK;
  API_END
}

extern "C" int ssamg_diffusion_exp_gradient(ssamg_solver s, const double* g, const double* lambda,
                                            const double* x, double* dg, void* stream) {
  if (!s || !g || !lambda || !x || !dg) return SSAMG_ERR_ARG;
  if (!s->ready) return SSAMG_ERR_STATE;
  API_BEGIN
  // the kernel differentiates one box with the 7-point stencil's faces
  const Level& L0 = s->lev[0];
  if (L0.np != 1)
    throw SsamgError{SSAMG_ERR_UNSUPPORTED, "the diffusion gradient takes a grid of one part"};
  {
    const PartH& h = L0.parts[0];
    int seen = 0;
    bool ok = h.nent == 7;
    for (int e = 0; e < h.nent && ok; ++e) {
      const int a = std::abs(h.o[e][0]) + std::abs(h.o[e][1]) + std::abs(h.o[e][2]);
      if (a > 1) ok = false;
      else seen |= 1 << ((h.o[e][0] + 1) + 3 * (h.o[e][1] + 1) + 9 * (h.o[e][2] + 1));
    }
    if (!ok || seen != ((1 << 4) | (1 << 10) | (1 << 12) | (1 << 13) | (1 << 14) | (1 << 16) |
                        (1 << 22)))
      throw SsamgError{SSAMG_ERR_UNSUPPORTED, "the diffusion gradient needs the 7-point stencil"};
  }
  PdlScope pdl(s->prm);
  // kappa = exp(g) goes to the PCG's q vector (scratch between solves)
  launch_diffusion_exp_gradient(s->lev[0], g, lambda, x, dg, s->q, (cudaStream_t)stream);
  return SSAMG_OK;
  API_END
}

extern "C" int ssamg_precondition(ssamg_solver s, const double* r, double* z, void* stream) {
  if (!s || !r || !z) return SSAMG_ERR_ARG;
  if (!s->ready) return SSAMG_ERR_STATE;
  API_BEGIN
  PdlScope pdl(s->prm);
  vcycle(s, r, z, (cudaStream_t)stream);
  return SSAMG_OK;
  API_END
}

extern "C" int ssamg_level_matvec(ssamg_solver s, int level, const double* x, double* y,
                                  void* stream) {
  if (!s || !x || !y) return SSAMG_ERR_ARG;
  if (!s->ready) return SSAMG_ERR_STATE;
  if (level < 0 || level >= (int)s->lev.size()) return SSAMG_ERR_ARG;
  API_BEGIN
  PdlScope pdl(s->prm);
  launch_matvec(s->lev[level], x, y, (cudaStream_t)stream);
  return SSAMG_OK;
  API_END
}

// ---------------------------------------------------------------------------
// Batching form: independent problems as the parts of one system
// ---------------------------------------------------------------------------
struct ssamg_batch_s {
  int nprob = 0;
  ssamg_grid g = nullptr;
  ssamg_matrix A = nullptr;
  ssamg_solver s = nullptr;
  std::vector<long long> off;  // nprob + 1 first unknowns
  ~ssamg_batch_s() {
    ssamg_solver_destroy(s);
    ssamg_matrix_destroy(A);
    ssamg_grid_destroy(g);
  }
};

namespace {
void check(int rc) {
  if (rc != SSAMG_OK) throw SsamgError{rc, g_last_error};
}
}  // namespace

extern "C" int ssamg_batch_create(int nprob, const ssamg_matrix* A, const ssamg_params* prm,
                                  void* stream, ssamg_batch* out) {
  if (!out || !A || nprob < 1) return SSAMG_ERR_ARG;
  for (int k = 0; k < nprob; ++k) {
    if (!A[k]) return SSAMG_ERR_ARG;
    if (!A[k]->assembled) return SSAMG_ERR_STATE;
  }
  const ssamg_matrix A0 = A[0];
  for (int k = 1; k < nprob; ++k) {
    if (A[k]->g->ndim != A0->g->ndim || A[k]->nent != A0->nent) return SSAMG_ERR_UNSUPPORTED;
    for (int e = 0; e < A0->nent; ++e)
      for (int d = 0; d < 3; ++d)
        if (A[k]->o[e][d] != A0->o[e][d]) return SSAMG_ERR_UNSUPPORTED;
  }
  API_BEGIN
  std::unique_ptr<ssamg_batch_s> B(new ssamg_batch_s);
  B->nprob = nprob;
  int total = 0;
  B->off.assign(nprob + 1, 0);
  for (int k = 0; k < nprob; ++k) {
    total += A[k]->g->nparts;
    B->off[k + 1] = B->off[k] + A[k]->g->N;
  }
  // union grid: the problems' parts in problem order
  check(ssamg_grid_create(A0->g->ndim, total, &B->g));
  std::vector<int> part_prob;
  part_prob.reserve(total);
  for (int k = 0, P = 0; k < nprob; ++k) {
    const ssamg_grid g = A[k]->g;
    for (int q = 0; q < g->nparts; ++q, ++P) {
      check(ssamg_grid_set_box(B->g, P, g->lo[q].data(), g->hi[q].data()));
      part_prob.push_back(k);
    }
  }
  check(ssamg_grid_assemble(B->g));
  // union matrix: the same stencil; values copied part by part (device to
  // device), couplings with their parts renumbered
  std::vector<int> offs(3 * A0->nent);
  for (int e = 0; e < A0->nent; ++e)
    for (int d = 0; d < 3; ++d) offs[3 * e + d] = A0->o[e][d];
  check(ssamg_matrix_create(B->g, A0->nent, offs.data(), &B->A));
  for (int k = 0, P = 0; k < nprob; ++k) {
    const ssamg_matrix M = A[k];
    for (int q = 0; q < M->g->nparts; ++q, ++P)
      for (int e = 0; e < M->nent; ++e) {
        if (M->isvar[q][e])
          check(ssamg_matrix_set_box_values(B->A, P, e, M->coef + M->coef_off[q][e], 1));
        else
          check(ssamg_matrix_set_constant(B->A, P, e, M->cval[q][e]));
      }
    // couplings: the problem's cells shifted by its first cell in the union
    const long long nc = (long long)M->c_val.size();
    if (nc > 0) {
      ssamg_matrix U = B->A;
      const int shift = (int)B->off[k];
      for (long long t = 0; t < nc; ++t) {
        U->c_row.push_back(M->c_row[t] + shift);
        U->c_col.push_back(M->c_col[t] + shift);
      }
      U->c_bits.insert(U->c_bits.end(), M->c_bits.begin(), M->c_bits.end());
      U->c_val.insert(U->c_val.end(), M->c_val.begin(), M->c_val.end());
      U->c_hasu.resize(B->g->nparts, 0);
      const int p0 = P - M->g->nparts;
      for (int q = 0; q < M->g->nparts && q < (int)M->c_hasu.size(); ++q)
        U->c_hasu[p0 + q] = std::max(U->c_hasu[p0 + q], M->c_hasu[q]);
      U->assembled = false;
    }
  }
  check(ssamg_matrix_assemble(B->A, stream));
  check(ssamg_solver_create(prm, &B->s));
  B->s->nprob = nprob;
  B->s->part_prob = std::move(part_prob);
  *out = B.release();
  return SSAMG_OK;
  API_END
}

extern "C" int ssamg_batch_setup(ssamg_batch B, void* stream) {
  NvtxRange nv("ssamg_batch_setup");
  if (!B) return SSAMG_ERR_ARG;
  return ssamg_setup(B->s, B->A, stream);
}

extern "C" long long ssamg_batch_num_cells(ssamg_batch B) { return B ? B->off.back() : -1; }

extern "C" int ssamg_batch_offsets(ssamg_batch B, long long* off) {
  if (!B || !off) return SSAMG_ERR_ARG;
  std::copy(B->off.begin(), B->off.end(), off);
  return SSAMG_OK;
}

extern "C" int ssamg_batch_solve(ssamg_batch B, const double* b, double* x, int nrhs, void* stream,
                                 ssamg_stats* st) {
  NvtxRange nv("ssamg_batch_solve");
  if (!B || !b || !x || nrhs < 1) return SSAMG_ERR_ARG;
  ssamg_solver s = B->s;
  if (!s->ready) return SSAMG_ERR_STATE;
  cudaStream_t cst = (cudaStream_t)stream;
  API_BEGIN
  PdlScope pdl(s->prm);
  if (s->prm.use_graph) return run_rounds(s, b, x, nrhs, cst, st);
  const long long N = s->lev[0].N;
  int rc = SSAMG_OK;
  for (int j = 0; j < nrhs; ++j) {
    SSAMG_CUDA(cudaMemcpyAsync(s->b, b + j * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, cst));
    SSAMG_CUDA(cudaMemsetAsync(s->x, 0, sizeof(double) * N, cst));
    const int r = run_pcg(s, cst, st ? st + (long long)j * B->nprob : nullptr);
    SSAMG_CUDA(cudaMemcpyAsync(x + j * N, s->x, sizeof(double) * N, cudaMemcpyDeviceToDevice, cst));
    if (r < 0) return r;
    if (r > rc) rc = r;
  }
  return rc;
  API_END
}

extern "C" ssamg_solver ssamg_batch_solver(ssamg_batch B) { return B ? B->s : nullptr; }

extern "C" void ssamg_batch_destroy(ssamg_batch B) { delete B; }

// ---------------------------------------------------------------------------
// Introspection
// ---------------------------------------------------------------------------
extern "C" int ssamg_num_parts(ssamg_solver s) {
  return (s && s->ready) ? s->lev[0].np : SSAMG_ERR_STATE;
}

extern "C" int ssamg_tail_levels(ssamg_solver s, int* first, int* ctas, long long* smem_bytes) {
  if (!s || !s->ready) return SSAMG_ERR_STATE;
  const bool on = s->ctail_lt >= 1;
  if (first) *first = on ? s->ctail_lt : -1;
  if (ctas) *ctas = on ? s->ctail_nc : 0;
  if (smem_bytes) *smem_bytes = on ? s->ctail_smem : 0;
  return on ? s->ctail.nt : 0;
}

extern "C" int ssamg_num_levels(ssamg_solver s) {
  return (s && s->ready) ? (int)s->lev.size() : SSAMG_ERR_STATE;
}

extern "C" int ssamg_level_part_info(ssamg_solver s, int level, int part, int* lo, int* hi,
                                     int* dstar, double* omega, int* nentries, int* offsets,
                                     long long* cell_offset) {
  if (!s || !s->ready) return SSAMG_ERR_STATE;
  if (level < 0 || level >= (int)s->lev.size()) return SSAMG_ERR_ARG;
  const Level& L = s->lev[level];
  if (part < 0 || part >= L.np) return SSAMG_ERR_ARG;
  const PartH& h = L.parts[part];
  for (int d = 0; d < 3; ++d) {
    if (lo) lo[d] = h.lo[d];
    if (hi) hi[d] = h.hi[d];
  }
  if (dstar) *dstar = h.dstar;
  if (omega) *omega = h.omega;
  if (nentries) *nentries = h.nent;
  if (offsets)
    for (int e = 0; e < h.nent; ++e)
      for (int d = 0; d < 3; ++d) offsets[3 * e + d] = h.o[e][d];
  if (cell_offset) *cell_offset = h.off;
  return SSAMG_OK;
}

extern "C" int ssamg_level_sizes(ssamg_solver s, int level, long long* ncells, long long* u_rows,
                                 long long* u_nnz) {
  if (!s || !s->ready) return SSAMG_ERR_STATE;
  if (level < 0 || level >= (int)s->lev.size()) return SSAMG_ERR_ARG;
  const Level& L = s->lev[level];
  if (ncells) *ncells = L.N;
  if (u_rows) *u_rows = L.nr;
  if (u_nnz) *u_nnz = L.nnz;
  return SSAMG_OK;
}

extern "C" int ssamg_level_copy(ssamg_solver s, int level, int what, int part, int entry, void* dst,
                                long long n) {
  if (!s || !s->ready) return SSAMG_ERR_STATE;
  if (!dst || level < 0 || level >= (int)s->lev.size()) return SSAMG_ERR_ARG;
  const Level& L = s->lev[level];
  API_BEGIN
  auto copy = [&](const void* src, size_t bytes, long long want) {
    argcheck(n == want, "destination size does not match the data size");
    if (want == 0) return;
    argcheck(src != nullptr, "no such data on this level");
    SSAMG_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
  };
  auto part_ok = [&]() { argcheck(part >= 0 && part < L.np, "part out of range"); };
  switch (what) {
    case 0: {
      part_ok();
      const PartH& h = L.parts[part];
      argcheck(entry >= 0 && entry < h.nent, "entry out of range");
      if (h.var[entry]) {
        copy(L.coef + h.coef_off[entry], sizeof(double) * h.ncell, h.ncell);
      } else {
        argcheck(n == h.ncell, "destination size does not match the data size");
        std::fill((double*)dst, (double*)dst + n, h.cval[entry]);
      }
      break;
    }
    case 1:
    case 2: {
      part_ok();
      const PartH& h = L.parts[part];
      argcheck(h.dstar >= 0, "part is not coarsened at this level");
      copy((what == 1 ? L.Pw : L.Pe) + h.poff, sizeof(double) * h.nfine, h.nfine);
      break;
    }
    case 3: copy(L.dinv, sizeof(double) * L.N, L.N); break;
    case 4: copy(L.u_ptr, sizeof(int) * (L.nr + 1), L.nr > 0 ? L.nr + 1 : 0); break;
    case 5: copy(L.u_rows, sizeof(int) * L.nr, L.nr); break;
    case 6: copy(L.u_col, sizeof(int) * L.nnz, L.nnz); break;
    case 7: copy(L.u_val, sizeof(double) * L.nnz, L.nnz); break;
    case 8: copy(L.u_bits, (size_t)L.nnz, L.nnz); break;
    default: return SSAMG_ERR_ARG;
  }
  return SSAMG_OK;
  API_END
}

extern "C" int ssamg_level_stored_coefficients(ssamg_solver s, int level, long long* ncoef) {
  if (!s || !ncoef) return SSAMG_ERR_ARG;
  if (!s->ready) return SSAMG_ERR_STATE;
  if (level < 0 || level >= (int)s->lev.size()) return SSAMG_ERR_ARG;
  *ncoef = s->lev[level].ncoef;
  return SSAMG_OK;
}

extern "C" int ssamg_spacings(ssamg_solver s, double* c, double* W) {
  if (!s || !s->ready) return SSAMG_ERR_STATE;
  if (c) std::copy(s->c.begin(), s->c.end(), c);
  if (W) std::copy(s->W.begin(), s->W.end(), W);
  return SSAMG_OK;
}

extern "C" int ssamg_coupling_sums_noalloc(ssamg_solver s, int level, double* c_dev,
                                           void* stream) {
  if (!s || !c_dev) return SSAMG_ERR_ARG;
  if (!s->ready) return SSAMG_ERR_STATE;
  API_BEGIN
  argcheck(level >= 0 && level < (int)s->lev.size(), "level out of range");
  const Level& L = s->lev[level];
  if (L.nblk > SSAMG_NOALLOC_MAX_BLOCKS) {
    char msg[160];
    std::snprintf(msg, sizeof msg,
                  "coupling sums of level %d need %d blocks of scratch; the static scratch holds %d",
                  level, L.nblk, SSAMG_NOALLOC_MAX_BLOCKS);
    throw SsamgError{SSAMG_ERR_UNSUPPORTED, msg};
  }
  launch_wsum(L, noalloc_scratch(), c_dev, (cudaStream_t)stream);
  return SSAMG_OK;
  API_END
}

// Times one hot-path kernel: `reps` launches captured into a CUDA graph,
// replayed once to warm up and once between events on `stream`.
// Mean microseconds per launch of `reps` launches of one kernel, captured
// into a graph and replayed (after one warm-up replay) between events on st.
// The caller has checked the arguments and set the launch scope.
double time_kernel_us(ssamg_solver s, int kernel, int level, int reps, cudaStream_t st) {
  if (!s->cs) SSAMG_CUDA(cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking));
  Level& L = s->lev[level];
  const bool f = s->prm.precision == 1;
  auto one = [&](cudaStream_t cs) {
    switch (kernel) {
      case 0:  // residual r = b - A x
        if (f) launch_residual<float>(L, (const float*)L.x, (const float*)L.b, (float*)L.r, cs);
        else launch_residual<double>(L, (const double*)L.x, (const double*)L.b, (double*)L.r, cs);
        break;
      case 1:  // relaxation t = x + omega M^-1 (b - A x)
        if (f) launch_relax<float>(L, (const float*)L.x, (const float*)L.b, (float*)L.t, cs);
        else launch_relax<double>(L, (const double*)L.x, (const double*)L.b, (double*)L.t, cs);
        break;
      case 2:  // pre-relaxation from zero with U x
        if (f) launch_relax0_u<float>(L, (const float*)L.b, (float*)L.x, cs);
        else launch_relax0_u<double>(L, (const double*)L.b, (double*)L.x, cs);
        break;
      case 3:  // restriction to level + 1
        // with the next level's pre-relaxation, as the cycle runs it
        if (f)
          launch_restrict<float>(L, s->lev[level + 1], (const float*)L.r, (float*)s->lev[level + 1].b,
                                 level + 2 < (int)s->lev.size() ? (float*)s->lev[level + 1].x : nullptr, cs);
        else
          launch_restrict<double>(L, s->lev[level + 1], (const double*)L.r,
                                  (double*)s->lev[level + 1].b,
                                  level + 2 < (int)s->lev.size() ? (double*)s->lev[level + 1].x : nullptr, cs);
        break;
      case 4:  // prolongation from level + 1 with U x
        if (f) launch_prolong_u<float>(L, (const float*)s->lev[level + 1].x, (const float*)L.x, (float*)L.r, cs);
        else launch_prolong_u<double>(L, (const double*)s->lev[level + 1].x, (const double*)L.x, (double*)L.r, cs);
        break;
      case 5:  // whole V-cycle
        vcycle(s, s->r, s->z, cs);
        break;
      case 6:  // FP64 operator apply of the PCG (q = A p with p.q partials)
        launch_pcg_alpha(s->lev[0], s->p, s->q, pcg_ctx(s), cs);
        break;
      case 7:  // one PCG iteration (V-cycle, beta, p, q = A p, alpha, x and r)
        enqueue_pcg_body(s, 0, 0, cs);
        break;
      case 9:  // the cycle's last post-relaxation as the PCG runs it (FP64 z, dot partials)
        if (f)
          launch_relax_final<float>(s->lev[0], (const float*)s->lev[0].r,
                                    (const float*)s->lev[0].b, s->z, s->r, s->prm.flexible ? s->zprev : nullptr,
                                    s->partial, cs);
        else
          launch_relax_final<double>(s->lev[0], (const double*)s->lev[0].r,
                                     (const double*)s->lev[0].b, s->z, s->r,
                                     s->prm.flexible ? s->zprev : nullptr, s->partial, cs);
        break;
      case 8:  // the PCG's vector steps: beta, p = z + beta p, alpha, x and r updates
        launch_pcg_beta_from_partials(s->lev[0], s->z, s->p, pcg_ctx(s),
                                      final_ranges(s->lev[0], pcg_ctx(s)), cs);
        launch_pcg_update(s->lev[0], s->p, s->q, s->x, s->r, pcg_ctx(s), 0, 0, cs);
        break;
      case 10: {  // the coarse-level transition's cluster kernel (levels from ctail_lt on)
        if (s->ctail_lt < 1) throw SsamgError{SSAMG_ERR_STATE, "no cluster tail in this hierarchy"};
        Level& T0 = s->lev[s->ctail_lt];
        if (f)
          launch_ctail<float>(s->ctail, s->ctail_nc, s->ctail_smem, (const float*)T0.b, (float*)T0.t, cs);
        else
          launch_ctail<double>(s->ctail, s->ctail_nc, s->ctail_smem, (const double*)T0.b,
                               (double*)T0.t, cs);
        break;
      }
      case 11:    // residual of every right-hand side of the last batch solve, one launch
      case 12: {  // relaxation likewise (cell-tile levels above the tail)
        const RhsSet& M = s->rhs;
        if (M.R < 2 || level >= M.nlev || uses_bricks(L))
          throw SsamgError{SSAMG_ERR_STATE, "no right-hand sides solved together on this level"};
        const RhsSaved saved = save_rhs(s);
        SkipScope none(nullptr);
        use_rhs(s, 0);
        g_ssamg_skip = nullptr;  // every instance takes part
        const long long vs = M.stride[level];
        if (kernel == 11) {
          if (f) launch_residual_rhs<float>(L, M.R, vs, s->nprob, (const float*)L.x, (const float*)L.b, (float*)L.r, cs);
          else launch_residual_rhs<double>(L, M.R, vs, s->nprob, (const double*)L.x, (const double*)L.b, (double*)L.r, cs);
        } else {
          if (f) launch_relax_rhs<float>(L, M.R, vs, s->nprob, (const float*)L.x, (const float*)L.b, (float*)L.t, cs);
          else launch_relax_rhs<double>(L, M.R, vs, s->nprob, (const double*)L.x, (const double*)L.b, (double*)L.t, cs);
        }
        restore_rhs(s, saved);
        break;
      }
      default:
        throw SsamgError{SSAMG_ERR_ARG, "unknown kernel id"};
    }
  };
  if (kernel == 7 || kernel == 8) {
    // keep the iteration from stopping: no convergence test, no iteration cap
    SSAMG_CUDA(cudaMemcpyAsync(s->h_sc, s->sc, sizeof(PcgScalars) * s->nprob,
                               cudaMemcpyDeviceToHost, st));
    SSAMG_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < s->nprob; ++k) {
      s->h_sc[k].done = 0;
      s->h_sc[k].status = 0;
      s->h_sc[k].tol2bb = -1.0;
      s->h_sc[k].max_iter = 1 << 30;
    }
    SSAMG_CUDA(cudaMemcpyAsync(s->sc, s->h_sc, sizeof(PcgScalars) * s->nprob,
                               cudaMemcpyHostToDevice, st));
  }
  cudaGraph_t g;
  SSAMG_CUDA(cudaStreamBeginCapture(s->cs, cudaStreamCaptureModeThreadLocal));
  for (int t = 0; t < reps; ++t) one(s->cs);
  SSAMG_CUDA(cudaStreamEndCapture(s->cs, &g));
  cudaGraphExec_t ge;
  SSAMG_CUDA(cudaGraphInstantiate(&ge, g, 0));
  cudaGraphDestroy(g);
  cudaEvent_t e0, e1;
  SSAMG_CUDA(cudaEventCreate(&e0));
  SSAMG_CUDA(cudaEventCreate(&e1));
  SSAMG_CUDA(cudaGraphLaunch(ge, st));
  SSAMG_CUDA(cudaEventRecord(e0, st));
  SSAMG_CUDA(cudaGraphLaunch(ge, st));
  SSAMG_CUDA(cudaEventRecord(e1, st));
  SSAMG_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  SSAMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(ge);
  return 1e3 * ms / reps;
}

extern "C" int ssamg_time_kernel(ssamg_solver s, int kernel, int level, int reps,
                                 double* us_per_launch, void* stream) {
  if (!s || !us_per_launch || reps < 1) return SSAMG_ERR_ARG;
  if (!s->ready) return SSAMG_ERR_STATE;
  const int Lc = (int)s->lev.size() - 1;
  if (level < 0 || level > Lc || ((kernel == 3 || kernel == 4) && level >= Lc)) return SSAMG_ERR_ARG;
  API_BEGIN
  PdlScope pdl(s->prm);
  *us_per_launch = time_kernel_us(s, kernel, level, reps, (cudaStream_t)stream);
  return SSAMG_OK;
  API_END
}

// ------------------------------------------------------------- tile tuning

extern "C" int ssamg_set_tile_table(ssamg_solver s, const int* table) {
  if (!s) return SSAMG_ERR_ARG;
  if (table)
    for (int c = 0; c < SSAMG_TILE_CLASSES; ++c)
      if (!valid_tile(table[c])) return SSAMG_ERR_ARG;
  for (int c = 0; c < SSAMG_TILE_CLASSES; ++c) s->tiles[c] = table ? table[c] : 0;
  return SSAMG_OK;
}

extern "C" int ssamg_get_tile_table(ssamg_solver s, int* table) {
  if (!s || !table) return SSAMG_ERR_ARG;
  std::copy(s->tiles, s->tiles + SSAMG_TILE_CLASSES, table);
  return SSAMG_OK;
}

extern "C" int ssamg_level_tile(ssamg_solver s, int level, int* cells_per_thread, int* bricks) {
  if (!s || !cells_per_thread || !bricks) return SSAMG_ERR_ARG;
  if (!s->ready) return SSAMG_ERR_STATE;
  if (level < 0 || level >= (int)s->lev.size()) return SSAMG_ERR_ARG;
  PdlScope pdl(s->prm);
  *cells_per_thread = s->lev[level].cpt;
  *bricks = uses_bricks(s->lev[level]) ? 1 : 0;
  return SSAMG_OK;
}

// Time (us) of the kernels whose tiles follow level l's tile form, as one
// PCG iteration runs them: the residual, post-relaxation and prolongation on
// l, the restriction onto l, and on level 0 the PCG's operator apply and
// vector steps (the pre-relaxation from zero runs on flat element tiles).
double level_tile_cost(ssamg_solver s, int l, int reps, cudaStream_t st) {
  const int Lc = (int)s->lev.size() - 1;
  double t = 0.0;
  if (l < Lc) {
    t += time_kernel_us(s, 0, l, reps, st);
    t += time_kernel_us(s, l == 0 ? 9 : 1, l, reps, st);
    t += time_kernel_us(s, 4, l, reps, st);
  }
  if (l > 0) t += time_kernel_us(s, 3, l - 1, reps, st);
  if (l == 0) {
    t += time_kernel_us(s, 6, 0, reps, st);
    t += time_kernel_us(s, 8, 0, reps, st);
  }
  return t;
}

// PCG state on which whole iterations can be timed: b = 1, x = 0, the head
// and two iterations (the vectors then hold what an iteration meets).
void prime_pcg(ssamg_solver s, cudaStream_t st) {
  const long long N = s->lev[0].N;
  launch_fill(s->b, N, 1.0, st);
  SSAMG_CUDA(cudaMemsetAsync(s->x, 0, sizeof(double) * N, st));
  SSAMG_CUDA(cudaMemcpyAsync(s->sc, s->sc_init, sizeof(PcgScalars) * s->nprob,
                             cudaMemcpyDeviceToDevice, st));
  enqueue_pcg_head(s, 0, 0, st);
  enqueue_pcg_body(s, 0, 0, st);
  enqueue_pcg_body(s, 0, 0, st);
}

extern "C" int ssamg_autotune(ssamg_solver s, int reps, void* stream, int* table) {
  if (!s || reps < 1) return SSAMG_ERR_ARG;
  if (!s->ready || !s->A) return SSAMG_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  int saved[SSAMG_TILE_CLASSES];
  std::copy(s->tiles, s->tiles + SSAMG_TILE_CLASSES, saved);
  API_BEGIN
  // on an error the solver keeps the table it had (and needs a new set-up)
  struct Restore {
    ssamg_solver s;
    const int* saved;
    bool keep = false;
    ~Restore() {
      if (!keep) std::copy(saved, saved + SSAMG_TILE_CLASSES, s->tiles);
    }
  } restore{s, saved};
  PdlScope pdl(s->prm);
  const int B = SSAMG_TILE_BRICKS;
  static const int cand[] = {1, 2, 4, 1 | B, 2 | B, 4 | B};
  const int nc = (int)(sizeof(cand) / sizeof(cand[0]));
  const int nl = (int)s->lev.size();
  std::vector<int> cls(nl);
  for (int l = 0; l < nl; ++l) cls[l] = tile_class(level_cells(s->lev[l]));
  std::vector<double> def(nl, HUGE_VAL), cost((size_t)nl * nc, HUGE_VAL);
  // the built-in rule everywhere (the reference point), then each form
  // everywhere; the hierarchy itself does not depend on the tiles
  for (int k = -1; k < nc; ++k) {
    for (int c = 0; c < SSAMG_TILE_CLASSES; ++c) s->tiles[c] = k < 0 ? 0 : cand[k];
    run_setup(s, st);
    if ((int)s->lev.size() != nl) throw SsamgError{SSAMG_ERR_STATE, "hierarchy depth changed"};
    prime_pcg(s, st);
    for (int l = 0; l < nl; ++l) {
      // a brick form on a level that cannot use bricks is its cell form
      if (k >= 0 && (cand[k] & B) && !uses_bricks(s->lev[l])) continue;
      const double t = level_tile_cost(s, l, reps, st);
      if (k < 0) def[l] = t;
      else cost[(size_t)l * nc + k] = t;
    }
  }
  // per size class, the form of least time on the class's largest level,
  // kept only when it beats the built-in rule by SSAMG_TUNE_MARGIN
  int out[SSAMG_TILE_CLASSES] = {};
  std::vector<char> seen(SSAMG_TILE_CLASSES, 0);
  for (int l = 0; l < nl; ++l) {
    if (seen[cls[l]]) continue;
    seen[cls[l]] = 1;
    int best = -1;
    double bt = def[l];
    for (int k = 0; k < nc; ++k)
      if (cost[(size_t)l * nc + k] < bt) bt = cost[(size_t)l * nc + (best = k)];
    if (best >= 0 && bt < SSAMG_TUNE_MARGIN * def[l]) out[cls[l]] = cand[best];
  }
  // the per-level sums ignore how the kernels overlap in the solve: a table
  // is kept only when a whole PCG iteration under it beats the built-in rule
  if (std::any_of(out, out + SSAMG_TILE_CLASSES, [](int t) { return t != 0; })) {
    auto iteration_us = [&](const int* tb) {
      std::copy(tb, tb + SSAMG_TILE_CLASSES, s->tiles);
      run_setup(s, st);
      prime_pcg(s, st);
      return time_kernel_us(s, 7, 0, reps, st);
    };
    const int builtin[SSAMG_TILE_CLASSES] = {};
    const double t0 = iteration_us(builtin);
    const double t1 = iteration_us(out);
    if (!(t1 < SSAMG_TUNE_ITER_MARGIN * t0)) std::fill(out, out + SSAMG_TILE_CLASSES, 0);
  }
  std::copy(out, out + SSAMG_TILE_CLASSES, s->tiles);
  run_setup(s, st);
  restore.keep = true;
  if (table) std::copy(out, out + SSAMG_TILE_CLASSES, table);
  return SSAMG_OK;
  API_END
}

extern "C" int ssamg_selftest_barrier(int nblocks, int extra_arrivals, unsigned max_polls,
                                      void* stream) {
  if (nblocks < 1 || nblocks > 8 || extra_arrivals < 0 || extra_arrivals > 1024 ||
      max_polls < 1 || max_polls > (1u << 20))
    return SSAMG_ERR_ARG;
  API_BEGIN
  const int err = barrier_selftest(nblocks, extra_arrivals, max_polls, (cudaStream_t)stream);
  if (err) throw SsamgError{SSAMG_ERR_TIMEOUT, "the grid barrier gave up after its poll cap"};
  return SSAMG_OK;
  API_END
}

extern "C" int ssamg_residual_history(ssamg_solver s, int problem, double* rel, int n) {
  if (!s || !rel || n < 0) return SSAMG_ERR_ARG;
  if (!s->ready) return SSAMG_ERR_STATE;
  if (problem < 0 || problem >= s->nprob) return SSAMG_ERR_ARG;
  API_BEGIN
  PcgScalars sc;
  SSAMG_CUDA(cudaMemcpy(&sc, s->sc + problem, sizeof(sc), cudaMemcpyDeviceToHost));
  const int stride = s->prm.max_iter + 1;
  const int m = std::min(n, std::min(sc.iter, s->prm.max_iter) + 1);
  if (m <= 0) return 0;
  std::vector<double> h((size_t)m);
  SSAMG_CUDA(cudaMemcpy(h.data(), s->hist + (long long)problem * stride, sizeof(double) * m,
                        cudaMemcpyDeviceToHost));
  for (int k = 0; k < m; ++k) rel[k] = sc.bb > 0 ? std::sqrt(h[k] / sc.bb) : 0.0;
  return m;
  API_END
}

extern "C" int ssamg_set_spacings(ssamg_solver s, int nparts, const double* W) {
  if (!s || nparts < 0) return SSAMG_ERR_ARG;
  if (!W || nparts == 0) {
    s->user_W.clear();
    return SSAMG_OK;
  }
  for (int t = 0; t < 3 * nparts; ++t)
    if (!(W[t] > 0.0)) return SSAMG_ERR_ARG;  // NaN, zero or negative
  s->user_W.assign(W, W + 3 * nparts);
  s->ready = false;
  return SSAMG_OK;
}

extern "C" int ssamg_selftest_fastdiv(unsigned long long seed, int trials) {
  // host check of the division constants against plain division
  unsigned long long z = seed;
  for (int t = 0; t < trials; ++t) {
    z = z * 6364136223846793005ull + 1442695040888963407ull;
    unsigned d = (unsigned)((z >> 33) % 4000000u) + 1u;
    z = z * 6364136223846793005ull + 1442695040888963407ull;
    unsigned n = (unsigned)(z >> 33) & 0x7fffffffu;
    FastDiv f = make_fastdiv(d);
    if (fdiv(n, f) != n / d) return 1;
    if (fdiv(d * (n / d), f) != n / d) return 2;
  }
  return 0;
}
