/*
 * ssamg.h - C ABI of a GB300 (sm_103a) implementation of the data-parallel
 * hot path of semi-structured algebraic multigrid (SSAMG; Magri, Falgout and
 * Yang, arXiv 2205.14273).
 *
 * Objects follow the paper's semi-structured interface (Section 2): a grid of
 * parts, each one logically rectangular box of cell-centred indices; a
 * stencil of offsets shared by the parts, whose coefficients are either
 * constant over a part or given per cell; and inter-part couplings (the
 * unstructured matrix U).  A = S + U.
 *
 * Conventions for every call:
 *  - Return value: SSAMG_OK (0) on success, SSAMG_NOT_CONVERGED (1) as a
 *    warning from the solves, a negative ssamg_status on failure.  A failed
 *    call leaves its objects unchanged unless stated otherwise.
 *  - Handles are opaque and owned by the library; *_destroy frees them.
 *  - Vectors are FP64, parts in order, each part's box with i fastest, then
 *    j, then k (N = total number of cells).  Pointers marked "device" are
 *    CUDA device pointers owned by the caller; they are read or written
 *    asynchronously on the given stream.  Pointers marked "host" are copied
 *    before the call returns.
 *  - stream: a cudaStream_t (NULL = legacy default stream).
 *  - Objects are not thread-safe; use one handle per host thread.
 */
#ifndef SSAMG_H
#define SSAMG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ssamg_grid_s* ssamg_grid;
typedef struct ssamg_matrix_s* ssamg_matrix;
typedef struct ssamg_solver_s* ssamg_solver;

typedef enum {
  SSAMG_OK = 0,
  SSAMG_NOT_CONVERGED = 1,   /* iteration limit reached; stats are filled in */
  SSAMG_ERR_ARG = -1,        /* invalid argument (index, size, box, offset) */
  SSAMG_ERR_STATE = -2,      /* call out of order (e.g. solve before setup) */
  SSAMG_ERR_OOM = -3,        /* device or host allocation failed */
  SSAMG_ERR_CUDA = -4,       /* a CUDA runtime call failed */
  SSAMG_ERR_BREAKDOWN = -5,  /* PCG breakdown (p.Ap <= 0, NaN/Inf) or a non-SPD coarsest operator */
  SSAMG_ERR_TIMEOUT = -6,    /* a bounded device wait gave up */
  SSAMG_ERR_UNSUPPORTED = -7 /* a size limit of this implementation was exceeded */
} ssamg_status;

/* Human-readable text for a status code (static storage). */
const char* ssamg_status_string(int status);
/* Detail of the last failure on the calling host thread (valid until the
 * next failing call on that thread). */
const char* ssamg_last_error(void);
/* Device memory and pinned host buffers that destroyed matrices and solvers
 * left to the library's pools (kept per rounded size and reused by the next
 * objects, so that creating them per step costs no cudaMalloc / cudaFree /
 * cudaMallocHost) are returned to the driver.  Returns the number of device
 * bytes released.  Never fails. */
long long ssamg_release_device_cache(void);

/* ---------------------------------------------------------------- grid ---
 * Section 2 (semi-structured grid): nparts parts with independent index
 * spaces.  ndim in {1,2,3}; unused dimensions must have lo = hi.
 * This implementation takes one box per part (the part's bounding box,
 * Section 3.1 footnote, is then the box itself). */
int ssamg_grid_create(int ndim, int nparts, ssamg_grid* out);
/* Inclusive lower and upper corners of the box of `part` (3 ints each). */
int ssamg_grid_set_box(ssamg_grid g, int part, const int lo[3], const int hi[3]);
/* Another box of `part` (after its ssamg_grid_set_box; Section 2: a part is
 * a group of boxes in one index space, at most 16).  The part is held over
 * the bounding box of its boxes: vectors and coefficient arrays of the part
 * cover the bounding box (i fastest); cells outside the boxes are decoupled
 * unknowns (diagonal 1, no stencil connection into or out of them, values
 * given for them ignored), so the solution there is the right-hand side's
 * value and every other cell is solved exactly as the group of boxes.
 * Stencil connections between the part's boxes are kept (interpolation
 * crosses them).  SSAMG_ERR_ARG for a box with hi < lo, before set_box or
 * after assemble; SSAMG_ERR_UNSUPPORTED beyond 16 boxes or 2^30 cells. */
int ssamg_grid_add_box(ssamg_grid g, int part, const int lo[3], const int hi[3]);
/* Checks that every part has a non-empty box; freezes the grid. */
int ssamg_grid_assemble(ssamg_grid g);
/* Total number of cells (valid after assemble), or -1. */
long long ssamg_grid_num_cells(ssamg_grid g);
void ssamg_grid_destroy(ssamg_grid g);

/* -------------------------------------------------------------- matrix ---
 * Section 2 (A = S + U).  offsets: nentries x 3 ints in {-1,0,1}, shared by
 * all parts (at most 27 entries, each offset at most once).  S(c, c+o) is the
 * entry's coefficient at c when c+o lies in the part's box and zero
 * otherwise: connections that leave a part are either a physical boundary
 * (eliminated) or part of U.  The matrix must be symmetric positive definite
 * for the solves; symmetry of U is the caller's duty. */
int ssamg_matrix_create(ssamg_grid g, int nentries, const int* offsets, ssamg_matrix* out);
/* Entry `entry` of part `part` is `value` at every cell. */
int ssamg_matrix_set_constant(ssamg_matrix A, int part, int entry, double value);
/* Entry `entry` of part `part` varies per cell: vals holds the part's cells
 * in vector order (i fastest).  vals_on_device: 0 = host pointer, 1 = device
 * pointer; the values are copied either way.  Values of connections that
 * leave the box are ignored. */
int ssamg_matrix_set_box_values(ssamg_matrix A, int part, int entry, const double* vals,
                                int vals_on_device);
/* Adds n couplings U(row, col) += vals[t] (host arrays, copied).  Row cell:
 * part[t], absolute index idx[3t..3t+2]; column cell: nbor_part[t],
 * nbor_idx[3t..3t+2].  dir[3t..3t+2] is the offset through which the row's
 * cell leaves its part toward the column (one component +-1 for a face
 * coupling; 0,0,0 for a non-geometric one); it marks the part boundaries that
 * interpolation must not cross (Section 3.2).  A row with a nonzero dir
 * leaves its part that way: the neighbour through dir lies outside the part
 * (outside its box, or outside the boxes of a part of several); a row with
 * dir 0,0,0 may lie anywhere in its part (e.g. beside ghost unknowns under a
 * refined patch, Section 4 test case 4).  Rows and columns lie in their
 * parts' boxes, columns in a different part.  Duplicates are summed. */
int ssamg_matrix_add_couplings(ssamg_matrix A, long long n, const int* part, const int* idx,
                               const int* dir, const int* nbor_part, const int* nbor_idx,
                               const double* vals);
/* Validates and uploads the matrix to the device (synchronous on stream). */
int ssamg_matrix_assemble(ssamg_matrix A, void* stream);
void ssamg_matrix_destroy(ssamg_matrix A);

/* -------------------------------------------------------------- solver --- */
typedef struct {
  int precision;       /* 0: FP64 V-cycle; 1: FP32 V-cycle inside FP64 PCG */
  int relax;           /* 0: weighted Jacobi (Eq. relax1); 1: L1 Jacobi (Section 3.4) */
  double relax_factor; /* <= 0: omega_p of Eq. relax1 (relax 0) or 3/2 (relax 1) */
  int skip;            /* Section 3.4 "skip" (relaxation turned off on some levels, mimicking
                          full coarsening).  0 (default): relax on every level.  1: per part,
                          the levels form rounds of distinct coarsening directions (a round
                          starts at level 0 and wherever d* repeats a direction of the current
                          round); only the first level of each round relaxes, so an isotropic
                          part (d*_l = d*_{l-n_d}) relaxes on levels 0, n_d, 2 n_d, ... and a
                          part coarsened repeatedly along one direction keeps relaxing there
                          (Section 4, test case 2); levels where the part is not coarsened
                          relax.  2: the printed test alone: no relaxation at level l >= n_d
                          when d*_l = d*_{l-n_d} */
  int max_levels;      /* l_max of Section 3.1 (default 64) */
  long long s_max;     /* coarsening stops at total size <= s_max; <= 0: number of parts */
  double tol;          /* PCG stop: ||r||_2 <= tol ||b||_2 (default 1e-8) */
  int max_iter;        /* PCG iteration limit (default 200) */
  int coarse_direct;   /* 1: dense Cholesky on the coarsest level; 0: one relaxation sweep (Section 3.5) */
  int flexible;        /* 1: Polak-Ribiere beta (for the FP32 cycle); 0: Fletcher-Reeves */
  int use_graph;       /* 1: run the PCG iteration loop as one CUDA graph */
  int use_tail;        /* coarse levels in one launch: 0 one launch per level and step;
                          1: a cooperative grid over the levels of at most 32,768 cells
                          (<= 8 parts), with grid barriers; 2: one CTA of 1024 threads over the
                          levels of at most tail_cells cells (<= 8 parts), with block barriers;
                          3 (default): the coarse-level transition of Section 3.5 (hybrid
                          idea): from the
                          first level of at most tail_cells cells (default 4096) down, the
                          levels are assembled at setup (A = S + U as CSR, P, P^T, smoother
                          diagonal, coarsest inverse) and each V-cycle runs them in one
                          thread-block cluster with the level vectors in distributed shared
                          memory (the first tail level is lowered while the tail does not fit
                          the cluster's shared memory; no tail of two or more levels: as 0) */
  int use_pdl;         /* 1 (default): launch the solve's kernels with programmatic dependent
                          launch, so that each kernel is scheduled, and stages its part
                          descriptors, while its predecessor still runs; 0: plain launches */
  int tail_cells;      /* largest level of the use_tail = 2 or 3 tail (0: 4096) */
  int use_bricks;      /* 1 (default): residual, relaxations (also the last one, with the PCG's
                          dot partials) and PCG operator applies on checked 7-point levels
                          (some entries constant per part) run over 32 x 8 x 8 bricks, each
                          thread marching a column along z; 0: over the cell tiles of the
                          other shapes */
  int rhs_together;    /* ssamg_batch_solve with several right-hand sides and use_graph:
                          1 (default) one PCG loop for all of them, each cycle step enqueued
                          per right-hand side except the residual and relaxation on cell-tile
                          levels, which take every right-hand side in one launch (the blocks
                          of a tile side by side, so its stencil coefficients are read from
                          HBM once); 0: the right-hand sides one after another in one graph.
                          Both give the same results; a hierarchy with the fused tail of
                          use_tail 1 or 2 always takes 0 */
} ssamg_params;

typedef struct {
  int iterations;
  int converged;
  double rel_res;       /* ||r_k|| / ||b|| of the recursive residual */
  double true_rel_res;  /* ||b - A x|| / ||b|| recomputed at exit (FP64) */
  int num_levels;
  long long coarse_size;
  double operator_complexity; /* sum of stored stencil+U entries over levels / level 0 */
  long long setup_kernel_launches;  /* kernels launched by the last ssamg_setup */
  long long solve_kernel_launches;  /* kernels run by the PCG of this right-hand side */
} ssamg_stats;

/* Fills *p with the defaults listed above. */
void ssamg_params_default(ssamg_params* p);
int ssamg_solver_create(const ssamg_params* p, ssamg_solver* out);
void ssamg_solver_destroy(ssamg_solver s);

/* Builds the hierarchy (Sections 3.1-3.4): per-part coupling sums and
 * spacings W, Algorithm 1, interpolation (Eq. prolEx), Galerkin coarse
 * operators (Eq. galerkin) and relaxation diagonals, then factors the
 * coarsest operator.  The matrix must stay alive until the solver is
 * destroyed or set up again.  Synchronises `stream`. */
int ssamg_setup(ssamg_solver s, ssamg_matrix A, void* stream);

/* PCG preconditioned by one V(1,1) cycle (Section 4), x0 = 0 when
 * zero_guess != 0, else x holds x0.  b, x: device, nrhs vectors of N
 * doubles each.  With use_graph and nrhs > 1, all right-hand sides run in
 * one graph launch as ssamg_batch_solve runs them (rhs_together); else one
 * after another.  Stops at ||r|| <= tol ||b||.  st may be NULL (stats of
 * the last right-hand side). */
int ssamg_solve(ssamg_solver s, const double* b, double* x, int nrhs, int zero_guess,
                void* stream, ssamg_stats* st);
/* Same as ssamg_solve with host b and x; the copies are part of the call. */
int ssamg_solve_host(ssamg_solver s, const double* b, double* x, int nrhs, void* stream,
                     ssamg_stats* st);
/* Adjoint solve A^T lambda = g with the forward hierarchy (A is symmetric,
 * so A^T = A and the same V-cycle applies).  g, lambda: device. */
int ssamg_adjoint_solve(ssamg_solver s, const double* g, double* lambda, int nrhs, void* stream,
                        ssamg_stats* st);
/* dL/da_e(c) = -lambda_c x_{c+o_e} for every entry e and cell c (zero where
 * c+o_e leaves the box): the gradient of L(x(A)) with respect to the level-0
 * stencil coefficients, given lambda = A^-T dL/dx.  lambda, x: device, N
 * doubles.  dcoef: device, nentries x N doubles (entry-major). */
int ssamg_coef_gradient(ssamg_solver s, const double* lambda, const double* x, double* dcoef,
                        void* stream);
/* dL/dg for the 7-point harmonic-mean diffusion operator with kappa = exp(g)
 * on one part (off-diagonal -2 k_c k_n/(k_c+k_n), diagonal = sum |off| + k_c
 * per Dirichlet face): dL/dg_c = k_c (sum over interior faces of
 * -2 k_n^2/(k_c+k_n)^2 (lam_c - lam_n)(x_c - x_n) - lam_c x_c per Dirichlet
 * face).  g, lambda, x, dg: device, N doubles.  The solver's grid must have
 * one part and its stencil the seven 7-point offsets (any order), else
 * SSAMG_ERR_UNSUPPORTED before anything is enqueued.
 * exp(g) is formed once per cell in the solver's PCG work vector q, which
 * the next solve overwrites anyway. */
int ssamg_diffusion_exp_gradient(ssamg_solver s, const double* g, const double* lambda,
                                 const double* x, double* dg, void* stream);

/* One V(1,1) cycle z = M r (device pointers; in the solver's precision). */
int ssamg_precondition(ssamg_solver s, const double* r, double* z, void* stream);
/* y = A_l x on level l (FP64, device pointers of the level's size). */
int ssamg_level_matvec(ssamg_solver s, int level, const double* x, double* y, void* stream);

/* ------------------------------------------------------- introspection ---
 * For tests and diagnostics (host copies; synchronous). */
int ssamg_num_levels(ssamg_solver s);
/* Coarse-level transition of use_tail = 3: returns the number of levels it
 * runs (0: none), with its first level, the CTAs of its cluster and their
 * shared memory in bytes (-1, 0, 0 when there is none).  SSAMG_ERR_STATE
 * before setup.  Any output pointer may be NULL. */
int ssamg_tail_levels(ssamg_solver s, int* first, int* ctas, long long* smem_bytes);
/* Number of parts of the set-up hierarchy (every level has the same parts);
 * SSAMG_ERR_STATE before setup. */
int ssamg_num_parts(ssamg_solver s);
/* Per level and part: box corners, d* (-1 when the part is not coarsened or
 * on the coarsest level), omega_p (Eq. relax1), number of stencil entries and
 * their offsets (nentries x 3 ints, up to 27), offset of the part in the
 * level vector.  Any output pointer may be NULL. */
int ssamg_level_part_info(ssamg_solver s, int level, int part, int* lo, int* hi, int* dstar,
                          double* omega, int* nentries, int* offsets, long long* cell_offset);
/* Level size and number of U rows and nonzeros. */
int ssamg_level_sizes(ssamg_solver s, int level, long long* ncells, long long* u_rows,
                      long long* u_nnz);
/* Copies level data to host memory:
 *  what 0: stencil coefficients of (part, entry): ncells(part) doubles
 *  what 1: P west weights of part (fine points only, see below)
 *  what 2: P east weights of part
 *  what 3: smoother diagonal omega M^-1 of the whole level (N_l doubles)
 *  what 4: U row pointers (u_rows+1 ints)   what 5: U row cells (u_rows ints)
 *  what 6: U column cells (u_nnz ints)       what 7: U values (u_nnz doubles)
 *  what 8: U direction bits (u_nnz bytes)
 * The P weights of a coarsened part are stored for its fine points only: the
 * box with its d* extent replaced by (n + p) / 2 (p = lo[d*] mod 2), cell
 * (..., F, ...) being fine cell 2F + 1 - p along d*.  n is the number of
 * elements the destination holds; it must equal the data size. */
int ssamg_level_copy(ssamg_solver s, int level, int what, int part, int entry, void* dst,
                     long long n);
/* Number of stored per-cell stencil coefficients of a level (constant
 * entries excluded), for algorithmic-byte counts. */
int ssamg_level_stored_coefficients(ssamg_solver s, int level, long long* ncoef);
/* Residual history of the last solved right-hand side of `problem` (0 for a
 * single system; a batch's problem index otherwise): rel[k] = ||r_k|| / ||b||
 * of the PCG's recursive residual for k = 0 .. iterations, at most n values
 * (host array).  Returns the number written (>= 0), or SSAMG_ERR_STATE
 * before a setup, SSAMG_ERR_ARG for a bad problem index or pointer.  Call
 * once the solve's stream has completed (synchronous copies). */
int ssamg_residual_history(ssamg_solver s, int problem, double* rel, int n);

/* Representative grid spacings given by the user (Section 3.1: an option
 * PFMG offers, used only for coarsening): W is n_parts x 3 host doubles
 * (part-major, x y z), each > 0 (+inf: never coarsen along that dimension;
 * unused dimensions are ignored), copied.  From the next ssamg_setup on,
 * Algorithm 1 and the relaxation weights of Eq. relax1 take them instead of
 * the spacings computed from the coupling sums; W = NULL (or nparts = 0)
 * returns to the computed ones.  SSAMG_ERR_ARG for a NaN, zero or negative
 * value; the next setup fails with SSAMG_ERR_ARG when nparts does not match
 * the matrix's grid. */
int ssamg_set_spacings(ssamg_solver s, int nparts, const double* W);

/* Per-part coupling sums c (n_parts x 3) and spacings W (n_parts x 3) of
 * Section 3.1 (W = +inf encoded as HUGE_VAL). */
int ssamg_spacings(ssamg_solver s, double* c, double* W);

/* ---------------------------------------------------------------------------
 * Batching form (not in the paper, whose solver handles one system): many
 * independent problems, and several right-hand sides each, solved together.
 * The problems' parts become the parts of one semi-structured system with no
 * couplings between problems.  One setup then builds every problem's
 * hierarchy at once (Algorithm 1 and the Galerkin products act part by part;
 * the parts of a problem that reaches one cell per part early stay through
 * the remaining levels, where P is the identity and the coarsest direct solve
 * stays exact), and every cycle kernel covers all problems in one launch per
 * level.  PCG (Section 4) runs one instance per problem: its own dot
 * products, step sizes and stopping test, until every problem has stopped.
 * ------------------------------------------------------------------------- */
typedef struct ssamg_batch_s* ssamg_batch;

/* Batch of nprob assembled matrices, each on its own grid; all share the
 * grid dimension and the stencil (same entries in the same order), else
 * SSAMG_ERR_UNSUPPORTED.  Values and couplings are copied, so the matrices
 * may be destroyed afterwards.  prm as for ssamg_solver_create (one setting
 * for all problems).  Synchronises `stream`. */
int ssamg_batch_create(int nprob, const ssamg_matrix* A, const ssamg_params* prm, void* stream,
                       ssamg_batch* out);
/* Builds the hierarchies of all problems (ssamg_setup on the union). */
int ssamg_batch_setup(ssamg_batch B, void* stream);
/* N, the number of unknowns of all problems together (-1 for NULL). */
long long ssamg_batch_num_cells(ssamg_batch B);
/* off[0..nprob]: the first unknown of each problem in a batch vector
 * (off[nprob] = N); problem k's unknowns are in its own grid's order. */
int ssamg_batch_offsets(ssamg_batch B, long long* off);
/* Solves A_k x_kj = b_kj for every problem k and right-hand side j from
 * x0 = 0.  b, x: device, nrhs x N doubles (right-hand side j at j N).
 * st: NULL or nrhs x nprob stats, entry j nprob + k.  Returns SSAMG_OK when
 * every instance converged, SSAMG_NOT_CONVERGED when one hit max_iter, else
 * the first error.  With use_graph, all right-hand sides run in one graph
 * launch (together or one after another, see rhs_together) and `stream` is
 * synchronised once; without, once per right-hand side.  The residual
 * history (ssamg_residual_history) is the last right-hand side's. */
int ssamg_batch_solve(ssamg_batch B, const double* b, double* x, int nrhs, void* stream,
                      ssamg_stats* st);
/* The solver the batch runs on (owned by the batch), for the introspection
 * and timing calls (ssamg_num_levels, ssamg_level_sizes, ssamg_time_kernel
 * ...); NULL for NULL. */
ssamg_solver ssamg_batch_solver(ssamg_batch B);
void ssamg_batch_destroy(ssamg_batch B);

/* Blocks whose partial sums fit the static scratch of
 * ssamg_coupling_sums_noalloc: 3 doubles each, 1.5 MiB of device memory.
 * Under the built-in tile rule a level launch covers 1024 cells per block
 * when the level has 300,000 cells or more (256 below), so levels of up to
 * 67,108,864 cells fit (fewer under a tile table of fewer cells per thread). */
#define SSAMG_NOALLOC_MAX_BLOCKS 65536

/* Allocation-free form of the per-part coupling sums: for each part and
 * dimension d, the sum over the part's cells of sign(a_C) times minus the
 * stencil entries whose offset moves along d, for level `level` of a set-up
 * hierarchy.  The paper has no counterpart: this variant exists for callers
 * that cannot allocate device memory where they call it (inside a captured
 * CUDA graph, or under an allocator they do not control), so it takes no
 * memory and never synchronises.
 *   c_dev  device, n_parts(level) x 3 doubles, caller-owned; on level 0 it
 *          receives the values ssamg_spacings reports, bit for bit.
 *   stream stream the two kernels are enqueued on; the call returns without
 *          waiting.
 * Block partials go to one fixed static device array of
 * SSAMG_NOALLOC_MAX_BLOCKS x 3 doubles.  A level that needs more blocks is
 * rejected with SSAMG_ERR_UNSUPPORTED (the message in ssamg_last_error
 * gives both counts) before anything is enqueued.  Nothing in the scratch
 * needs to start at zero: every block writes its own partials before the
 * final sums read them.  ssamg_setup resolves the scratch address once per
 * device (outside any capture); later calls make no CUDA runtime call that
 * is illegal during stream capture.  The scratch is shared by every solver
 * on the device: two calls that may run at the same time (streams with no
 * ordering between them, or host threads) race on it and give wrong sums. */
int ssamg_coupling_sums_noalloc(ssamg_solver s, int level, double* c_dev, void* stream);

/* Diagnostic timing of one hot-path kernel on `level`: `reps` launches are
 * captured into a CUDA graph and replayed between CUDA events on `stream`
 * (after one warm-up replay); *us_per_launch receives the mean time per launch
 * in microseconds.  kernel: 0 residual, 1 relaxation, 2 pre-relaxation from
 * zero (with U x; the cycle runs it on level 0 only), 3 restriction to level+1
 * (with level+1's pre-relaxation when level+1 is not the coarsest, as the
 * cycle runs it), 4 prolongation from level+1 (with U x), 5 whole V-cycle
 * (level ignored), 6 the PCG's FP64 level-0 operator apply with its dot
 * product (level ignored), 7 one whole PCG iteration, 8 the PCG's vector steps
 * (beta, search direction, alpha, x and r updates), 9 the cycle's last post-
 * relaxation as the PCG runs it (FP64 z out, r.z partials), 10 the coarse-level transition's
 * cluster kernel of use_tail = 3 (level ignored; SSAMG_ERR_STATE without one), 11 and 12 the
 * residual and the relaxation of every right-hand side of the last batch solve in one launch
 * (rhs_together; cell-tile levels above the tail, SSAMG_ERR_STATE elsewhere).  Ids 7 and 8 clear
 * the solve's convergence state, so that the replayed iterations never stop,
 * and run on the vectors the last solve left (time them after a solve: on
 * vectors that break the iteration down, p.Ap <= 0, the cycle kernels stand
 * idle); the next solve starts afresh.  The kernels work on the solver's own
 * buffers (their contents are overwritten).  Synchronises `stream`.
 */
int ssamg_time_kernel(ssamg_solver s, int kernel, int level, int reps, double* us_per_launch,
                      void* stream);

/* ---------------------------------------------------------- tile forms ---
 * The paper has no counterpart: this is how the kernels map threads to cells.
 * Every per-level launch covers the level's cells in one tile form, chosen
 * per level from its cell count n (summed over parts):
 *   k cells per thread (k = 1 .. 4): blocks of 256 threads over 256 k
 *     consecutive cells of one part, a thread's cells 256 apart;
 *   bricks (on levels whose operator is the 7-point stencil with some
 *     entries constant per part, use_bricks set): the residual, relaxations
 *     and PCG operator applies run over 32 x 8 x 8 bricks, each thread
 *     marching a column along z; the other kernels keep the cell tiles.
 * The tile table has one entry per size class c = floor(log2(max(n, 1))),
 * c = 0 .. SSAMG_TILE_CLASSES - 1: 0 selects the built-in rule (4 cells per
 * thread from 300,000 cells up, 1 below; bricks where the level allows
 * them), k alone selects k cells per thread without bricks, and
 * k | SSAMG_TILE_BRICKS k cells per thread with bricks allowed.  A tile form
 * decides only which thread computes which cell: every cycle result is the
 * same bit for bit under any table; the PCG's dot products, summed per
 * block, round differently. */
#define SSAMG_TILE_CLASSES 32
#define SSAMG_TILE_BRICKS 8

/* Sets the solver's tile table from table[SSAMG_TILE_CLASSES] (copied), or
 * clears it to the built-in rule (table NULL).  It applies from the next
 * ssamg_setup.  SSAMG_ERR_ARG (table unchanged) on an entry that is not 0,
 * k or k | SSAMG_TILE_BRICKS with 1 <= k <= 4.  Host only. */
int ssamg_set_tile_table(ssamg_solver s, const int* table);
/* Copies the solver's tile table into table[SSAMG_TILE_CLASSES].  Host only. */
int ssamg_get_tile_table(ssamg_solver s, int* table);
/* The tile form level `level` of the set-up hierarchy runs with: cells per
 * thread, and 1 in *bricks when its operator applies run over bricks.
 * Host only. */
int ssamg_level_tile(ssamg_solver s, int level, int* cells_per_thread, int* bricks);
/* Tile autotuner: a grid search over the forms {1, 2, 4} cells per thread,
 * each with and without bricks.  For each form, applied to every level, it
 * sets the hierarchy up again from the matrix of the last ssamg_setup and
 * times per level (as ssamg_time_kernel does, `reps` launches per kernel)
 * the kernels whose tiles follow that level's form: residual,
 * post-relaxation and prolongation on the level, restriction onto it, and
 * on level 0 the PCG's operator apply and vector steps (on PCG vectors
 * primed by two iterations for b = 1).  Per size class it keeps the fastest
 * form on the class's largest level when that saves at least 3% against the
 * built-in rule (else 0); a table with any entry set is then kept only if a
 * whole PCG iteration (ssamg_time_kernel id 7) under it is at least 1%
 * faster than under the built-in rule, else the table is all 0.  The table
 * is stored in the solver, the hierarchy set up once more with it, and
 * copied to table (SSAMG_TILE_CLASSES ints, or NULL).  Requires a set-up
 * solver; runs on `stream` and synchronises it; the set-ups reuse the
 * solver's device memory; the solver's PCG vectors are overwritten.  On an
 * error the solver keeps its previous table and must be set up again before
 * the next solve. */
int ssamg_autotune(ssamg_solver s, int reps, void* stream, int* table);

/* Self-test of the bounded device wait (the grid barrier of the cooperative
 * coarse-level kernel, use_tail = 1): nblocks (1..8) blocks of one
 * cooperative launch meet at one barrier that also waits for
 * extra_arrivals (0..1024) arrivals that never come; each waiting block
 * polls at most max_polls (1..2^20) times, then gives up and returns.
 * SSAMG_OK when the barrier completed (extra_arrivals = 0),
 * SSAMG_ERR_TIMEOUT when a block gave up; the device stays usable either
 * way.  SSAMG_ERR_ARG outside the ranges.  Synchronises `stream`. */
int ssamg_selftest_barrier(int nblocks, int extra_arrivals, unsigned max_polls, void* stream);

/* Host-only check of the run-time division constants the kernels use to
 * split a linear cell index into (i, j, k): compares against plain division
 * for `trials` pseudo-random (n, d) pairs.  Returns 0 when all agree. */
int ssamg_selftest_fastdiv(unsigned long long seed, int trials);

#ifdef __cplusplus
}
#endif
#endif /* SSAMG_H */
