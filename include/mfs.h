/*
 * mfs.h - C ABI of libmfs, a single-GPU (GB300, sm_103a) solver for monolithic
 * n-field coupled linear systems with block preconditioners.
 *
 * Problem (Sec. 4, the blocked system): A x = b with A = [A_ij], i, j = 1..N,
 * where A_ij couples field i (rows) to field j (columns) and any block may be
 * zero.  The solver is right-preconditioned flexible GMRES(m) (Sec. 3.1-3.2)
 * with one of three block preconditioners:
 *   MFS_BGS_AMG  block Gauss-Seidel with one smoothed-aggregation AMG V-cycle
 *                per diagonal block (Sec. 4.1);
 *   MFS_SIMPLE   n-field SIMPLE(AMG): fields merged into a predictor group and a
 *                Schur group, SIMPLEC / diagonal approximation of the predictor
 *                block, explicit approximate Schur complement (Sec. 4.2); a
 *                multi-field predictor group is solved by one BGS(AMG) sweep
 *                or, with simple_pred = MFS_PRED_AMG_BGS, by one monolithic
 *                AMG(BGS) V-cycle (SIMPLE(BGS(AMG)) / SIMPLE(AMG(BGS)) of
 *                Sec. 6.3); a Schur group at or below coarse_max dofs is
 *                solved directly by the dense LU of S~ (Sec. 6.3: a
 *                constraint block with a zero diagonal block);
 *   MFS_AMG_BGS  monolithic AMG with block-diagonal transfers, blockwise
 *                Galerkin coarse blocks and block Gauss-Seidel level smoothing
 *                (Sec. 4.3);
 *   MFS_BGS_GS   single-level BGS(GS): block Gauss-Seidel whose block solves
 *                are gs_sweeps multicolour Gauss-Seidel sweeps on the fine
 *                diagonal blocks (the paper's BGS(DD(GS)) comparison, Sec. 7.1,
 *                on one subdomain); requires smoother = MFS_GS;
 *   MFS_AMG_SIMPLE the same monolithic V-cycle with a SIMPLE step as level
 *                smoother (Sec. 4.3): per level, one BGS sweep of the
 *                single-field smoothers over the predictor fields, one
 *                smoother application on the explicit level Schur complement
 *                S~^l (one Schur field), then the SIMPLE update.
 * Every solve-phase step runs in this library's CUDA kernels; there is no CPU
 * fallback.  The AMG setup (strength graph, aggregation, tentative and
 * smoothed prolongators, Galerkin products, power iteration) runs in this
 * library's CUDA kernels too (the dense LU of the coarsest level, at most a
 * few hundred unknowns, is factored on the host) and is timed apart; a
 * host-only setup path computes the same hierarchy without a GPU.
 *
 * Each GMRES iteration (preconditioner, matvec, CGS2 Arnoldi, readback of
 * the Hessenberg column) is captured once per Krylov index into a CUDA graph
 * and replayed; a NULL params.cuda_stream makes the library create its own
 * (non-blocking) stream, which waits for the legacy default stream's earlier
 * work at the start of every call.
 *
 * Conventions
 *   - All functions return MFS_OK (0) or a negative MFS_ERR_* code;
 *     mfs_strerror() names it.  A failed call leaves no partial handle.
 *   - Vectors are float64, field-major: the vector of field 0, then field 1, ...
 *     Inside a field the dofs of a node are contiguous (dof = node * b + c).
 *   - Vector arguments may be host or device (CUDA) pointers; the library
 *     detects which and copies host data through its own device buffers.
 *   - Input block matrices are HOST pointers and are deep-copied; the caller
 *     may free them after mfs_setup returns.
 *   - Work is issued on params.cuda_stream (0 = legacy default stream); every
 *     call returns after its work on that stream has finished.
 *   - A handle is not thread-safe: one thread at a time per handle.
 */
#ifndef MFS_H
#define MFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MFS_MAX_FIELDS 8

enum mfs_status {
  MFS_OK = 0,
  MFS_ERR_INVALID = -1,        /* bad argument, shape or parameter */
  MFS_ERR_CUDA = -2,           /* CUDA runtime error or no usable GPU */
  MFS_ERR_OOM = -3,            /* device allocation failed */
  MFS_ERR_SINGULAR = -4,       /* zero pivot / zero diagonal in setup */
  MFS_ERR_NOT_CONVERGED = -5,  /* max_iters reached; x holds the last iterate */
  MFS_ERR_BREAKDOWN = -6,      /* non-finite value met inside GMRES */
  MFS_ERR_SETUP = -7           /* aggregation could not coarsen a field */
};

enum mfs_precond { MFS_BGS_AMG = 0, MFS_SIMPLE = 1, MFS_AMG_BGS = 2, MFS_AMG_SIMPLE = 3, MFS_BGS_GS = 4 };
enum mfs_bgs_order { MFS_BWD = 0, MFS_FWD = 1, MFS_SYM = 2 };
enum mfs_nullspace { MFS_NS_CONST = 0, MFS_NS_RBM = 1, MFS_NS_USER = 2 };
enum mfs_precision { MFS_FP64 = 0, MFS_FP32P = 1 };
enum mfs_simple_approx { MFS_ABSROWSUM = 0, MFS_DIAG = 1 };
enum mfs_smoother { MFS_CHEBYSHEV = 0, MFS_JACOBI = 1, MFS_GS = 2 };
enum mfs_simple_pred { MFS_PRED_BGS_AMG = 0, MFS_PRED_AMG_BGS = 1 };

/* One nonzero block A_ij as node-level block-CSR (BSR): nbrows x nbcols node
 * blocks of br x bc scalars (br = dofs per node of field i, bc = of field j),
 * block k holds vals[k*br*bc .. (k+1)*br*bc) row-major; colind sorted within
 * each row.  Host pointers. */
typedef struct {
  int i, j;
  int br, bc;
  int64_t nbrows, nbcols, nnzb;
  const int32_t *rowptr; /* nbrows + 1 */
  const int32_t *colind; /* nnzb */
  const double *vals;    /* nnzb * br * bc */
} mfs_block;

/* One physical field.  coords (host, nnodes * dim, may be NULL for
 * MFS_NS_CONST) give the rigid-body modes of an MFS_NS_RBM field
 * (requires dofs_per_node == dim).  petrov_galerkin = 1 marks a
 * non-symmetric diagonal block (the paper's fluid field, Sec. 7.2): its
 * hierarchy takes Petrov-Galerkin transfers after Sala & Tuminaro (2008),
 * R != P^T (local damping parameters minimising ||A p_j|| in the D^-1 norm,
 * moved to the rows by a minimum; R from the same construction on A^T).
 * The near-nullspace of smoothed aggregation (Sec. 3.3: the vectors the
 * tentative prolongator reproduces) is the constants per dof
 * (MFS_NS_CONST), the rigid-body modes (MFS_NS_RBM, rotations about each
 * aggregate's centroid) or the caller's vectors (MFS_NS_USER): ns_user
 * (host) holds ns_dim values per dof, dof-major (entry (d, q) at
 * ns_user[d * ns_dim + q], d = node * dofs_per_node + component), with
 * ns_dim and dofs_per_node in {1, 2, 3, 6}; the coarse levels have ns_dim
 * dofs per aggregate.  ns_user / ns_dim are ignored for the other kinds.
 * dirichlet (host, nnodes * dofs_per_node bytes, or NULL) flags dofs held by
 * Dirichlet conditions that the caller has eliminated: a flagged dof's row
 * must be the identity row across the field's block row (1 on the diagonal
 * of A_ii, 0 everywhere else; MFS_ERR_INVALID otherwise).  The fine level's
 * near-nullspace vectors are zero at flagged dofs (so the prolongator never
 * moves them), and a node whose every dof is flagged stays out of every
 * aggregate.  Copied by mfs_setup. */
typedef struct {
  int64_t nnodes;
  int dofs_per_node;
  int dim;
  const double *coords;
  int nullspace;          /* enum mfs_nullspace */
  double strength_theta;  /* strength-of-connection threshold, >= 0 */
  int petrov_galerkin;    /* 0: smoothed aggregation, R = P^T; 1: Petrov-Galerkin */
  const double *ns_user;  /* MFS_NS_USER: nnodes * dofs_per_node * ns_dim values */
  int ns_dim;             /* MFS_NS_USER: vectors in ns_user */
  const uint8_t *dirichlet; /* NULL or nnodes * dofs_per_node flags (nonzero: Dirichlet dof) */
} mfs_field;

typedef struct {
  int precond;                       /* enum mfs_precond */
  int bgs_order;                     /* enum mfs_bgs_order (default MFS_BWD) */
  int bgs_sweeps;                    /* k_max of BGS / SIMPLE (default 1) */
  int simple_group[MFS_MAX_FIELDS];  /* per field: 0 = predictor, 1 = Schur */
  int simple_approx;                 /* enum mfs_simple_approx */
  int max_levels;                    /* multigrid levels incl. the finest (>= 1) */
  int64_t coarse_max;                /* stop coarsening at <= this many dofs per group */
  int smoother;                      /* enum mfs_smoother */
  int cheb_degree;                   /* Chebyshev degree (default 2) */
  double cheb_ratio;                 /* lower interval end = lambda / ratio (30) */
  double cheb_boost;                 /* upper interval end = boost * lambda (1.1) */
  double jacobi_omega;               /* damped-Jacobi weight (2/3) */
  int jacobi_sweeps;                 /* damped-Jacobi sweeps (1) */
  int restart;                       /* GMRES restart length m (default 50) */
  int max_iters;                     /* total GMRES iterations (default 1000) */
  int precision;                     /* enum mfs_precision */
  uint64_t seed;                     /* SplitMix64 seed: priorities, power iteration */
  void *cuda_stream;                 /* cudaStream_t or NULL */
  int verbose;                       /* 0 = silent */
  int setup_only;                    /* 1: build the host hierarchy only (no GPU needed);
                                        the handle then serves the export calls alone */
  int profile;                       /* 1: time every kernel launch of mfs_solve with CUDA
                                        events, by kernel class (see mfs_kernel_stats) */
  int no_graphs;                     /* 1: launch kernels one by one instead of replaying
                                        one captured CUDA graph per GMRES iteration */
  int setup_device;                  /* 1 (default): AMG setup on the GPU; 0: on the host
                                        (C++/OpenMP); both compute the same hierarchy */
  int simple_pred;                   /* enum mfs_simple_pred: solver of SIMPLE's predictor
                                        group (default MFS_PRED_BGS_AMG) */
  int gs_sweeps;                     /* MFS_GS: sweeps per smoother application (1) */
  double gs_omega;                   /* MFS_GS: damping omega of the Gauss-Seidel update (0.79,
                                        the paper's DD(GS(0.79)), Sec. 7.1); 0 < omega < 2 */
  int rows_split;                    /* threads per block row of the float64 coupled matvec
                                        (merged row layout): 0 (default) = timed at setup
                                        among 1, 2 and 4; or 1, 2, 4 to fix it */
  int layout_tune;                   /* sparse layouts of matrices with >= 2048 block rows:
                                        0 (default) = the fastest of SELL-32 (2, 4 or 8
                                        slots in flight) and one warp per row, each timed
                                        alone (best for one solve at a time: a mid-size
                                        matrix cannot fill the GPU by itself); 1 = the same,
                                        but one warp per row only for rows of >= 32 blocks
                                        (best when many systems run together,
                                        mfs_solve_batch, where the GPU is full and
                                        throughput counts) */
  int vcycle_tail;                   /* 1: a single-field V-cycle whose level above the
                                        coarsest is small (<= 48 KB of vectors, one warp per
                                        block row, explicit coarse inverse) runs that level
                                        and the coarse solve as ONE single-CTA launch (same
                                        arithmetic, bit for bit); 0 (default): one launch per
                                        step (Algorithm 1 as written) - on GB300 the one-SM
                                        tail is no faster than the launches it replaces */
  int pdl;                           /* solve-phase kernels as programmatic dependent launches
                                        (each may be scheduled while its predecessor still
                                        runs and waits on the device for its results; the
                                        results are the same): 1 every launch, 0 none,
                                        N > 1 launches of at most N CTAs, -1 (default)
                                        while no other solve runs in the process: every
                                        launch of a system of at most 65,536 dofs (its
                                        kernels are too short to hide a launch), the
                                        launches of at most 160 CTAs of a larger one */
} mfs_params;

typedef struct {
  int iters;             /* preconditioner applications (GMRES iterations) */
  int restarts;
  int converged;         /* 1 when true residual <= tol */
  double true_relres;    /* ||b - A x|| / ||b - A x0||, float64, on the GPU */
  double est_relres;     /* GMRES (Givens) estimate at exit */
  double solve_ms;       /* wall time of mfs_solve */
  double setup_ms;       /* wall time of mfs_setup */
  int levels[2];         /* level count of hierarchy group 0 and 1 (or 0) */
} mfs_info;

/* Fill *p with the defaults listed above (BGS(AMG), backward, 1 sweep,
 * SIMPLE groups all zero = predictor is every field but the last, SIMPLEC, 4 levels, coarse_max 1000,
 * Chebyshev degree 2, GMRES(50), FP64, seed 7, GPU setup, V-cycle tails off). */
void mfs_default_params(mfs_params *p);

/* Build the hierarchy for the block system (Sec. 4: blocks A_ij with the
 * field map; Sec. 3.3 / 4.3: AMG setup and Galerkin coarse operators).
 * nblocks blocks with distinct (i, j); every diagonal block must be given.
 * On success *out owns all device data; free it with mfs_free. */
int mfs_setup(const mfs_block *blocks, int nblocks, const mfs_field *fields, int nfields,
              const mfs_params *params, struct mfs_handle **out);

/* Solve A x = rhs by FGMRES(m) to ||b - A x|| <= tol * ||b - A x0|| (Sec. 7.1
 * stopping rule) with x0 taken from x on entry.  rhs, x: n float64 (host or
 * device).  info may be NULL.  Returns MFS_ERR_NOT_CONVERGED with the last
 * iterate in x when max_iters is reached. */
int mfs_solve(struct mfs_handle *h, const double *rhs, double *x, double tol, mfs_info *info);

/* A new handle for the same system that shares `src`'s read-only device
 * hierarchy (matrices, transfers, smoother data, LU factors) and host copy,
 * with its own work vectors, Krylov basis, CUDA graphs and stream (`stream`,
 * or a new library-owned one when NULL).  Clones of one setup can solve
 * different right-hand sides at the same time (mfs_solve_batch).  The shared
 * data lives until the last of the handles is freed.  Profiling is off in
 * clones. */
int mfs_clone(const struct mfs_handle *src, void *stream, struct mfs_handle **out);

/* Solve nsys independent systems, one per handle (distinct handles; clones
 * of one setup allowed; any sizes, field counts, preconditioners and
 * precisions), each A_k x_k = rhs_k to tol as mfs_solve does; rhs / x host
 * or device.  Not in the paper: it batches many of the Sec. 3-4 solves.
 *  nthreads <= 0: fused.  The systems' FGMRES iterations advance together;
 *    every step of an iteration (each kernel of each system's preconditioner
 *    application, matvec and Arnoldi pass) runs as ONE launch over all
 *    systems of a group that take that kernel, driven by per-system argument
 *    tables, and the steps of an iteration are one CUDA graph replayed once
 *    per iteration on a library stream; systems that finish stop taking
 *    part.  The systems are split into -nthreads groups of similar sizes
 *    (0: one group per 32 systems, at most 8); each group's iterations are
 *    driven by its own host thread on its own library stream, so the groups
 *    progress independently.  A group's graph and tables are built on the
 *    first call with its handle list and kept for later calls with the same
 *    list (until one of its handles is freed).
 *  nthreads > 0: that many host threads each drive one handle's FGMRES at
 *    a time on the handle's own stream, so the systems' kernels overlap.
 * Either way every result is bit-for-bit the one mfs_solve gives for that
 * system alone.  infos / status (may be NULL) receive per-system results;
 * the return value is MFS_OK or the first failing system's code.  The
 * per-launch profiler is not used in batches. */
int mfs_solve_batch(struct mfs_handle *const *hs, int nsys, const double *const *rhs, double *const *x, double tol,
                    mfs_info *infos, int *status, int nthreads);

/* One preconditioner application z = M^-1 v (the Sec. 4 preconditioner with
 * x^(0) = 0 and k_max sweeps).  v, z: n float64, host or device. */
int mfs_apply(struct mfs_handle *h, const double *v, double *z);

/* y = A x with the fine coupled operator (all nonzero blocks), float64. */
int mfs_matvec(struct mfs_handle *h, const double *x, double *y);

/* *out = x . y for two device vectors of n float64 (n = mfs_ndofs), with
 * the solver's deterministic two-stage reduction (fixed per-block chunks,
 * then one block sums the partials; the Arnoldi dot products of Sec. 3.1's
 * GMRES use the same kernels).  The partial sums live in the handle's
 * device scratch.  Host pointers are rejected (MFS_ERR_INVALID). */
int mfs_dot(struct mfs_handle *h, const double *x, const double *y, double *out);

/* Measured float64 FMA rate of the current device, *tflops in TFLOP/s
 * (host).  The paper has no counterpart: it is the denominator of the
 * roofline of the float64 kernels (the coupled matvec and the Arnoldi
 * passes of Sec. 3.1's GMRES), which GB300's FP64 pipe bounds.  Launches
 * independent FMA chains on every SM on `stream` (NULL = legacy default
 * stream) in five launch shapes (8-32 chains per thread, 256-1024 threads
 * per CTA), timed by CUDA events, best rate after a warm-up; synchronous.
 * Errors: MFS_ERR_INVALID for a NULL output, MFS_ERR_CUDA. */
int mfs_fp64_rate(double *tflops, void *stream);

/* Allocation-free variant of mfs_dot.  The paper has no counterpart: it is
 * for callers that must not call cudaMalloc while they run - a host
 * framework whose caching allocator already holds the device memory, a
 * latency-critical loop that cannot take cudaMalloc's implicit device-wide
 * synchronisation, or a plug-in that may only allocate at initialisation.
 * *out (host) = x . y for device float64 vectors x, y of length n, computed
 * by the same two-stage reduction kernels as mfs_dot on `stream` (NULL =
 * legacy default stream) and synchronised before return; no handle needed.
 * The partial sums live in a static device array of
 * MFS_DOT_NOALLOC_PARTIALS + 32 doubles compiled into the library: every
 * device that loads the library holds it until the process exits.  The
 * call makes no cudaMalloc / cudaFree or other allocating call.  Its first
 * call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current.  The call synchronises
 * `stream`, so it cannot be made on a stream that is being captured (it is
 * refused there).  All calls share the one array: calls that overlap on the
 * GPU (other streams, other host threads) race, so serialise them.  Nothing
 * in the array needs clearing between calls.  Its launches are never
 * counted by the kernel statistics of a handle (mfs_kernel_stats), even
 * while another thread runs a profiled solve.
 * Errors: MFS_ERR_INVALID for NULL pointers, host vectors or vectors on
 * another device than the current one, a capturing stream, n < 0 or
 * n > MFS_DOT_NOALLOC_MAX_N (see mfs_last_error); MFS_ERR_CUDA when a CUDA
 * call fails. */
#define MFS_DOT_NOALLOC_PARTIALS 1024
#define MFS_DOT_NOALLOC_MAX_N ((int64_t)1 << 32)
int mfs_dot_noalloc(const double *x, const double *y, int64_t n, double *out, void *stream);

/* Total scalar dofs n of the coupled system. */
int64_t mfs_ndofs(const struct mfs_handle *h);

/* Device bytes held by the handle: shared != 0 -> the hierarchy shared with
 * its clones (matrices, transfers, LU factors); 0 -> its own workspace. */
int64_t mfs_device_bytes(const struct mfs_handle *h, int shared);

/* Export one hierarchy matrix as point CSR (float64) for inspection.
 * what: 0 = A block (i, j) of level, 1 = P of field i (level -> level+1),
 *       2 = R of field i.  group: 0 (all fields; SIMPLE: predictor group) or
 *       1 (SIMPLE Schur group, blocks of S~).  Call with NULL arrays to get
 *       *nrows, *ncols, *nnz; then with arrays of that size. */
int mfs_export_csr(const struct mfs_handle *h, int what, int group, int level, int i, int j,
                   int64_t *nrows, int64_t *ncols, int64_t *nnz,
                   int32_t *rowptr, int32_t *colind, double *vals);

/* Export per-level data.  what: 0 = aggregate id per node (int32, -1 for
 * unaggregated nodes), 1 = lambda_max estimate (1 double), 2 = SIMPLE
 * diagonal A~_11 of predictor field i (double, group 0; level 0 for
 * MFS_SIMPLE, level l for MFS_AMG_SIMPLE).  For MFS_AMG_SIMPLE, group 1
 * holds the level Schur complements S~^l (export_csr what 0, field 0) and
 * their lambda estimates.  3 = Gauss-Seidel colour per node (int32) of a
 * smoothed level (smoother MFS_GS): greedy first fit in node order, where
 * nodes i != j couple when an entry of block (i, j) or (j, i) exceeds 1e-12
 * times the largest entry of that block row.
 * cap = capacity in elements; *count receives the element count. */
int mfs_export_array(const struct mfs_handle *h, int what, int group, int level, int i,
                     void *buf, int64_t cap, int64_t *count);

/* Number of levels of hierarchy group g (0 when absent). */
int mfs_num_levels(const struct mfs_handle *h, int group);

/* Kernel accounting of the mfs_solve calls made since setup or the last
 * reset (handle built with params.profile = 1).  For class c in 0..4
 * (0 block SpMV incl. transfers, 1 fused smoothing step, 2 vector kernels,
 * 3 dense coarse solve, 4 Arnoldi reductions/updates) writes
 * out[3c] = launches, out[3c+1] = summed event time in ms,
 * out[3c+2] = summed algorithmic bytes (every matrix/vector entry a launch
 * touches counted once).  cap = length of out.  Returns the number of
 * classes written; reset != 0 zeroes the counters afterwards.  The event
 * hook is process-wide: profile one handle at a time. */
int mfs_kernel_stats(struct mfs_handle *h, double *out, int cap, int reset);

/* Per-kernel accounting behind mfs_kernel_stats: one row of 6 doubles per
 * kernel variant and size, sorted by summed time: [cls*100000 + sig, rows,
 * launches, ms, algorithmic bytes, algorithmic flops], where for SpMV (cls 0) and smoothing
 * (cls 1) sig = layout*1000 + br*100 + bc*10 + (float64 ? 1 : 0) with layout
 * 0 = SELL-32, 1 = warp-per-row BSR, 2 = merged coupled rows, 3 = SELL-32 with
 * 4 slots in flight (the layout autotuner's choices), and rows = block rows; for the other
 * classes sig is a kernel id and rows the vector length.  Returns the number
 * of rows written (cap = length of out).  Cleared by mfs_kernel_stats with
 * reset != 0. */
int mfs_kernel_detail(struct mfs_handle *h, double *out, int cap);

/* Record only the launches whose mfs_kernel_detail key equals `key` (and
 * whose row count equals `rows` unless rows == 0); key 0 records every
 * launch again.  Drops the captured iteration graphs so that they are
 * recaptured with the new set of timing events at the next solve.  Meant to
 * time one kernel inside a long run with little overhead. */
int mfs_profile_filter(struct mfs_handle *h, int key, int64_t rows);

/* Release every device and host resource of the handle (NULL is a no-op). */
void mfs_free(struct mfs_handle *h);
/* Static description of a status code. */
const char *mfs_strerror(int code);
/* Detail of the last failure on the calling thread ("" if none). */
const char *mfs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MFS_H */
