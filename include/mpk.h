/*
 * mpk.h - C ABI of the GB300 level-blocked matrix-power kernel library.
 *
 * The library computes the matrix-power kernel (MPK)
 *     y_0 = x,   y_k = A y_{k-1},   k = 1..p
 * for a square sparse matrix A (Sec. 3, first paragraph), using level-based
 * blocking (Sec. 4): a breadth-first search on the graph of A gives levels
 * (Eq. 3), rows are renumbered level by level, consecutive levels are
 * aggregated into level groups that fit the cache (Eq. 5), and a diagonal
 * wavefront over (level group, power) pairs (Fig. 5, with the point-to-point
 * conditions of Sec. 4.3) lets each slice of A be reused from on-chip memory
 * for several powers instead of being read from HBM p times.  It also runs
 * the Chebyshev time propagation built on the MPK (Sec. 7, Eq. 7-9).
 *
 * Conventions shared by every call:
 *  - Every call returns an mpk_status (0 = MPK_OK, negative = error) and
 *    never aborts the process.  mpk_strerror() names a status.
 *  - All matrix and vector pointers are DEVICE pointers on the current CUDA
 *    device unless a parameter says "host".  The caller owns them; the
 *    library never frees them and does not keep them after the call returns
 *    (mpk_plan copies what it needs).
 *  - The library owns a plan and all device memory inside it; release it
 *    with mpk_plan_destroy().
 *  - Work is ordered on the stream given in mpk_opts.stream (a cudaStream_t;
 *    NULL = the legacy default stream).  Calls that must report a
 *    device-side error synchronise that stream unless MPK_ASYNC is given.
 *  - Integers of the matrix are 32-bit (Fig. 1: int col[], rowPtr[]).
 *  - A plan is not thread-safe: calls on one plan must not overlap in time
 *    or on the GPU (they share the plan's dependency flags).
 */
#ifndef MPK_H
#define MPK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
typedef enum {
    MPK_OK = 0,
    MPK_ERR_INVALID = -1,     /* bad argument, or a malformed matrix          */
    MPK_ERR_CUDA = -2,        /* a CUDA runtime call failed                   */
    MPK_ERR_OOM = -3,         /* a device or host allocation failed           */
    MPK_ERR_TIMEOUT = -4,     /* a device-side dependency wait hit its limit  */
    MPK_ERR_UNSUPPORTED = -5  /* a valid request this build cannot serve      */
} mpk_status;

/* Storage / arithmetic precision of a plan.
 *  MPK_F64         matrix values, vectors and sums in FP64.
 *  MPK_F32         matrix values, vectors and sums in FP32.
 *  MPK_F32_BF16VAL vectors and sums in FP32; diagonal entries kept in FP32,
 *                  off-diagonal values stored as BF16 when every one of them
 *                  is exactly representable in BF16 (else FP32; see
 *                  mpk_plan_stats.val_bytes).
 *  MPK_F64_DF      FP64 vectors x and Y (same layouts and element type as
 *                  MPK_F64) with the arithmetic on the FP32 pipe in
 *                  double-float: every value is held as an unevaluated sum
 *                  hi + lo of two FP32 numbers (about 47 significant bits),
 *                  each row sum is a compensated dot product (exact products
 *                  by FMA, TwoSum of the partial sums, errors summed apart),
 *                  and each output element is rounded once to FP64.  Matrix
 *                  values are stored as FP32 when every one of them is
 *                  exactly an FP32 number (val_bytes 4), else as (hi, lo)
 *                  pairs (val_bytes 8).  The results of integer-valued
 *                  inputs are exact while they stay below 2^47 in magnitude.
 *                  Limits: block width nrhs = 1; every nonzero |a_ij| in
 *                  [2^-60, 2^60] (else mpk_plan returns MPK_ERR_UNSUPPORTED);
 *                  at run time max|x| * ||A||_inf^p must stay below 2^100
 *                  (else the call reports MPK_ERR_UNSUPPORTED and Y is not
 *                  valid); elements below 2^-100 in magnitude lose relative
 *                  precision (their absolute error stays below 2^-140).
 *                  mpk_run, mpk_run_host and mpk_baseline_run serve it (the
 *                  baseline with the same arithmetic, bit for bit); the
 *                  Chebyshev calls and batches return MPK_ERR_UNSUPPORTED.   */
typedef enum { MPK_F64 = 0, MPK_F32 = 1, MPK_F32_BF16VAL = 2, MPK_F64_DF = 3 } mpk_prec;

/* Tuning bits of mpk_opts.tune (for autotuners; 0 = defaults).
 *  MPK_TUNE_STAGE       stage each work item's matrix slice in shared memory
 *                       with bulk (TMA) copies, double-buffered, instead of
 *                       reading it from global memory (used when it fits).
 *  MPK_TUNE_EVICT_LAST  with staging: mark matrix slices evict-last in L2
 *                       until their last power (always evict-first then).  */
#define MPK_TUNE_STAGE      1u
#define MPK_TUNE_EVICT_LAST 2u
#define MPK_TUNE_NO_SORT    4u  /* keep rows in level order inside a tile even
                                   when sorting them by length (SELL-C-sigma,
                                   sigma = tile rows) would cut the padding   */
/*  MPK_TUNE_RESIDENT    each CTA owns a work item's tile for all p powers:
 *                       the tile's packed slice is copied into shared memory
 *                       once (bulk copies, two stages) and every power reads
 *                       it there, so the matrix leaves HBM once per sweep and
 *                       L2 carries only the vectors.  Tiles are sized to the
 *                       stage (tile_rows 0) and 1 or 2 CTAs run per SM
 *                       (ctas_per_sm).  Used when nrhs is 1 or 2, the stages
 *                       fit, and the grid exceeds (p-1) times the widest
 *                       forward dependency span in tiles (which rules out a
 *                       cycle of waits); otherwise the plan keeps the
 *                       work-list schedule (mpk_plan_stats.resident = 0).   */
#define MPK_TUNE_RESIDENT   8u

/* Flags of mpk_run / mpk_baseline_run / mpk_cheb. */
#define MPK_IO_PERMUTED 1u  /* x and outputs are in the plan's level order   */
#define MPK_ASYNC       2u  /* do not synchronise to read the device error word */
#define MPK_SWEEP_ONE   4u  /* mpk_cheb: one power per launch (back-to-back SpMVs,
                               the comparator of Sec. 7) instead of sweeps of p */

/* A square sparse matrix in CRS form (Sec. 3.1, Fig. 1).  Device pointers,
 * caller-owned.  rowptr[n+1] (rowptr[0] = 0, non-decreasing, rowptr[n] = nnz),
 * col[nnz] in [0, n), val[nnz] FP64 (col and val may be NULL when nnz = 0).
 * Column order inside a row is free.
 * assume_symmetric != 0 promises a structurally symmetric pattern; with 0 the
 * levels are computed on the pattern of A + A^T (Sec. 4 restricts the method
 * to symmetric patterns; the MPK itself always multiplies by A).          */
typedef struct {
    int32_t n;
    int64_t nnz;
    const int32_t *rowptr;
    const int32_t *col;
    const double *val;
    int32_t assume_symmetric;
} mpk_csr;

/* Planning options; initialise with mpk_opts_default().                  */
typedef struct {
    int32_t root;          /* BFS root vertex v_root (Sec. 4.1); default 0      */
    double cache_bytes;    /* C of Eq. 5 in bytes; 0 = the device's L2 size     */
    double safety_f;       /* f of Eq. 5; default 0.5 (Sec. 4.2.1)              */
    int32_t prec;          /* mpk_prec                                          */
    int32_t nrhs;          /* columns of the block vectors x, y_k (row-major)   */
    int32_t tile_rows;     /* rows per work item, multiple of 32; 0 = automatic */
    int32_t ctas_per_sm;   /* resident CTAs per SM of the wavefront; 0 = auto   */
    double timeout_s;      /* limit of every device-side wait; 0 = 2 seconds   */
    void *stream;          /* cudaStream_t for all work of this plan            */
    double lag;            /* extra slope of the wavefront: how many level groups
                              power k trails power k-1 beyond what the
                              dependencies need; < 0 = automatic (default)     */
    uint32_t tune;         /* MPK_TUNE_* bits                                   */
    int32_t recursion;     /* s_m of Sec. 4.4: maximum recursion stage (0 =
                              none, the default).  Runs of consecutive level
                              groups that violate Eq. 5 (one level each) are
                              refined by the BFS levels of the subgraph they
                              induce, rooted at the run's first row, and the
                              Eq. 5 groups of those sub-levels, stage after
                              stage; the issue order then places each item by
                              its latest dependency (the "diamond" of Sec. 4.4)
                              instead of one slope for all tiles.             */
    int32_t sweep;         /* powers per sweep, q (p_m of Eq. 5); 0 = p, the
                              default.  With q < p the issue order runs powers
                              1..q over all tiles in the wavefront order, then
                              q+1..2q, and so on, all in the one launch of
                              mpk_run: the first power of a sweep waits on the
                              flags of the last power of the one before, with
                              no launch boundary.  The level groups of Eq. 5
                              are sized for q powers (q = 1: power-major order,
                              p SpMVs chained by point-to-point flags).  The
                              resident schedule owns tiles for all p powers and
                              is not used when q < p.                         */
} mpk_opts;

/* Summary of a plan (all host values).                                    */
typedef struct {
    int32_t n, p, nrhs, prec;
    int64_t nnz;
    int32_t n_levels;      /* L_m                                                */
    int32_t n_groups;      /* number of level groups T(0..G-1)                   */
    int32_t n_tiles;       /* work items per power                               */
    int32_t max_level_rows;
    int32_t tile_rows;
    int32_t grid_ctas;     /* CTAs of the persistent wavefront launch            */
    int32_t val_bytes;     /* bytes per stored off-diagonal value (8, 4 or 2)    */
    int64_t packed_entries;/* stored entries incl. padding of the packed layout  */
    int64_t matrix_bytes;  /* device bytes of the packed matrix (values+indices) */
    int64_t device_bytes;  /* all device memory held by the plan                 */
    double plan_ms;        /* wall time of mpk_plan (phases in phase_ms)         */
    double cache_bytes;    /* C actually used in Eq. 5                           */
    double slope;          /* sigma: level groups between consecutive power fronts */
    int32_t staged;        /* 1 if work items stage their slice in shared memory */
    int32_t smem_bytes;    /* dynamic shared memory per wavefront CTA            */
    int32_t sorted;        /* 1 if rows are sorted by length inside each tile    */
    int32_t resident;      /* 1 if the plan runs the resident schedule           */
    int32_t dep_span;      /* widest forward dependency span, in tiles          */
    int32_t rec_stages;    /* recursion stages that refined something (Sec. 4.4) */
    int32_t sweep;         /* powers per sweep of the issue order (q <= p)       */
    double phase_ms[8];    /* wall time of mpk_plan by phase (sum = plan_ms):
                              [0] device attributes and CRS validation,
                              [1] transposed pattern and BFS levels,
                              [2] renumbering, P A P^T and row statistics,
                              [3] level sizes and precision checks,
                              [4] level groups (Eq. 5) and recursion,
                              [5] work items, packing, dependency ranges,
                              [6] grid size and issue order,
                              [7] flags, the last synchronisation and the
                                  release of temporary device memory        */
} mpk_plan_stats;

typedef struct mpk_plan_s *mpk_plan_t;

/* Fills *o with the defaults above.  MPK_ERR_INVALID if o is NULL.        */
int mpk_opts_default(mpk_opts *o);

/* Builds the level-blocked plan of A for powers 1..p (Sec. 4.5: the
 * preprocessing takes the matrix, p_m and C and yields the permutation).
 * On the GPU: validation, BFS levels (Eq. 3; when the search runs out of
 * vertices the lowest-numbered unvisited vertex starts the next level),
 * stable renumbering by (level, original index), the symmetric permutation
 * P A P^T, greedy level groups (Eq. 5, weight = stored entries x bytes per
 * entry of the chosen precision), the packed SELL-32 matrix (rows of a work
 * item sorted by length when that cuts the padding by more than 10%) and the
 * dependency ranges of the wavefront.  1 <= p <= 255, 1 <= nrhs <= 64.
 * Errors: MPK_ERR_INVALID (NULL rowptr, or NULL col / val with nnz > 0,
 * n < 1, p or nrhs out of range,
 * malformed CRS found on the device), MPK_ERR_OOM, MPK_ERR_CUDA.  On error
 * *out is set to NULL and nothing is leaked.                              */
int mpk_plan(const mpk_csr *A, int32_t p, const mpk_opts *o, mpk_plan_t *out);

/* Copies the plan summary to host memory *s.                              */
int mpk_plan_info(mpk_plan_t plan, mpk_plan_stats *s);

/* Matrix features for the learned planner (computed on the GPU while the
 * plan is built; HOST output out[count]): [0] log10 N, [1] mean and [2]
 * standard deviation of the stored entries per row, [3] log10(1 + longest
 * row), [4] mean and [5] maximum |column - row| / N of the level-ordered
 * matrix, [6] log10 L_m, [7] largest level / N, [8] mean / largest level size,
 * [9..24] share of the rows in each sixteenth of the level range.  Returns
 * the number of features (25), or MPK_ERR_INVALID.                        */
int mpk_plan_features(mpk_plan_t plan, float *out, int32_t count);

/* Copies plan arrays to caller-allocated DEVICE buffers; any may be NULL.
 *  perm[n]        perm[new] = old (Sec. 4.5: recovers the original order)
 *  level_ptr[L+1] first new row of each level (Fig. 3e); level_ptr[L] = n;
 *                 with recursion (Sec. 4.4) the finest levels: the levels
 *                 of the runs that were refined replaced by their sub-levels
 *  group_ptr[G+1] first level of each level group; group_ptr[G] = L
 *  level[n]       Eq. 3 level of each ORIGINAL vertex                      */
int mpk_plan_perm(mpk_plan_t plan, int32_t *perm, int32_t *level_ptr, int32_t *group_ptr,
                  int32_t *level);

/* The plan's schedule, copied to HOST arrays: work[n_tiles * p] = the issue
 * order of the work items, item = (tile << 8) | power; dep_lo / dep_hi
 * [n_tiles] = the range of tiles whose power k-1 a tile's power k waits for
 * (conditions (A)-(C) of Sec. 4.3 at tile granularity).  Every dependency of
 * an item precedes it in the order, which the in-order dealing of the
 * persistent launch relies on.  MPK_ERR_INVALID on NULL arguments.          */
int mpk_plan_schedule(mpk_plan_t plan, int32_t *work, int32_t *dep_lo, int32_t *dep_hi);

/* Level-blocked MPK (Sec. 4, Fig. 5 with level groups and point-to-point
 * synchronisation): Y[k-1] = A^k x for k = 1..p in ONE persistent launch.
 * x: n x nrhs row-major; Y: p consecutive blocks of n x nrhs.  Element type
 * double for MPK_F64, float otherwise.  Without MPK_IO_PERMUTED, x and Y are
 * in the caller's original numbering (the library gathers x and scatters Y
 * through a plan-owned buffer); with it, both are in the plan's level order
 * (new index r holds original vertex perm[r]), which is the fast path.
 * x and Y must not overlap.  Errors: MPK_ERR_INVALID, MPK_ERR_CUDA,
 * MPK_ERR_TIMEOUT (a wait exceeded opts.timeout_s; the outputs are then
 * incomplete), MPK_ERR_OOM (first unpermuted run on a large matrix).      */
int mpk_run(mpk_plan_t plan, const void *x, void *Y, uint32_t flags);

/* mpk_run with x and Y in HOST memory (same layouts and flags): x is copied
 * to the device, the level-blocked MPK runs, and each power is copied back
 * as soon as it is in the caller's numbering, its copy overlapping the
 * reordering of the next one.  Host memory should be page-locked
 * (cudaHostAlloc / cudaHostRegister, or a pinned torch tensor) for the
 * copies to run at link speed and overlap; pageable memory is accepted.
 * The copies use the plan's stream and a second stream of the plan; the
 * plan's stream waits for both, so with MPK_ASYNC synchronising the plan's
 * stream is enough before Y is read.  Device buffers are plan-owned
 * ((p + 3) blocks of n x nrhs elements, kept for later calls).  Errors as
 * mpk_run.                                                                 */
int mpk_run_host(mpk_plan_t plan, const void *x_host, void *Y_host, uint32_t flags);

/* Baseline MPK (Sec. 3.1, Fig. 1): p back-to-back SpMV launches over the
 * same packed matrix, y_k = A y_{k-1}.  Same arguments and results as
 * mpk_run; it is the comparator the level-blocked kernel is measured
 * against.                                                                */
int mpk_baseline_run(mpk_plan_t plan, const void *x, void *Y, uint32_t flags);

/* Gershgorin interval [lo, hi] of A (host outputs), from the plan's matrix:
 * lo = min_i (a_ii - sum_{j != i} |a_ij|), hi = max_i (a_ii + sum |a_ij|).
 * Used for the spectral scaling Ahat = (A - c)/r, c = (hi+lo)/2,
 * r = (hi-lo)/2, of the Chebyshev propagation (Sec. 7).                    */
int mpk_gershgorin(mpk_plan_t plan, double *lo, double *hi);

/* Host helper: the M+1 complex coefficients (interleaved re, im, HOST
 * memory) of exp(-i H dt) = sum_k coef_k T_k((H - c)/r) for the Schroedinger
 * equation (Sec. 7; Bessel-function coefficients, hbar = 1):
 * coef_0 = e^{-i c dt} J_0(r dt), coef_k = 2 e^{-i c dt} (-i)^k J_k(r dt).  */
int mpk_cheb_coeffs_schroedinger(int32_t M, double c, double r, double dt, double *coef);

/* Chebyshev time propagation (Sec. 7, Eq. 7-9) with the level-blocked MPK:
 *   Ahat = (A - c I)/r,  v_0 = x,  v_1 = Ahat v_0,  v_{k+1} = 2 Ahat v_k - v_{k-1},
 *   y = sum_{k=0}^{M} coef_k v_k,
 * where the M matrix applications run as ceil(M/p) wavefront sweeps of at
 * most p powers each (Sec. 7: M split into batches of p_m).  The plan must
 * have nrhs = 2: x and v_k are complex vectors stored as n x 2 (re, im) in
 * the plan precision (double for MPK_F64, float otherwise); y is n x 2
 * DOUBLE (the coefficient sum is accumulated in FP64).  coef: M+1 complex
 * numbers, interleaved, HOST memory.  Flags as for mpk_run, plus
 * MPK_SWEEP_ONE (same arithmetic, one power per launch).  Errors as for
 * mpk_run; MPK_ERR_INVALID if nrhs != 2, M < 1 or r == 0.                  */
int mpk_cheb(mpk_plan_t plan, const double *coef, int32_t M, double c, double r,
             const void *x, double *y, uint32_t flags);

/* Host helper: the M+1 real coefficients (HOST memory) of the heat-equation
 * propagator exp(-tau A) = sum_k coef_k T_k((A - c)/r), tau = a*dt (Sec. 7;
 * modified-Bessel coefficients): coef_0 = e^{-tau c} I_0(tau r),
 * coef_k = 2 e^{-tau c} (-1)^k I_k(tau r).  The scaled I_k(z) e^{-z} are
 * computed by Miller's backward recurrence normalised by
 * I_0 + 2 sum_k I_k = e^z.  MPK_ERR_INVALID if M < 0, r <= 0 or tau < 0.   */
int mpk_cheb_coeffs_heat(int32_t M, double c, double r, double tau, double *coef);

/* Host helper: the M+1 real coefficients (HOST memory) of A^{-1} =
 * sum_k coef_k T_k((A - c)/r) for a symmetric A with spectrum in
 * [c - r, c + r], c > r >= 0 (positive definite): with s = sqrt(c^2 - r^2)
 * and q = r / (c + s) < 1, coef_0 = 1/s and coef_k = 2 (-q)^k / s.  The
 * truncation after M terms errs by at most 2 q^{M+1} / (s (1 - q)) on the
 * interval.  With mpk_cheb_real this applies a polynomial approximation of
 * the inverse (a polynomial preconditioner, or a fixed-degree solve) in
 * MPK sweeps.  MPK_ERR_INVALID unless M >= 0 and c > r >= 0.               */
int mpk_cheb_coeffs_inverse(int32_t M, double c, double r, double *coef);

/* Real Chebyshev propagation (the heat equation of Sec. 7): as mpk_cheb with
 * a plan of nrhs = 1, x and v_k real vectors of n entries in the plan
 * precision, coef M+1 real numbers (HOST memory), and y n DOUBLES.
 * MPK_ERR_INVALID if nrhs != 1, M < 1 or r == 0.                           */
int mpk_cheb_real(mpk_plan_t plan, const double *coef, int32_t M, double c, double r,
                  const void *x, double *y, uint32_t flags);

/* Several time steps of the Chebyshev propagation (Sec. 7) in one call:
 * y = U^nsteps x with U = sum_{k=0}^{M} coef_k T_k((A - c)/r), complex
 * (plan nrhs = 2; coef: M+1 complex numbers, interleaved) or real (plan
 * nrhs = 1; coef: M+1 reals), layouts and flags as mpk_cheb /
 * mpk_cheb_real.  The nsteps*M matrix applications run as wavefront sweeps
 * of the plan's p powers that continue across the time steps: the node of a
 * step's last power hands its row of the step's result, in the storage
 * precision, to the next step as v_0, so a plan with p >= nsteps*M runs the
 * whole propagation in one launch.  Results equal nsteps calls of
 * mpk_cheb / mpk_cheb_real whose x is the previous y in the storage
 * precision.  MPK_ERR_INVALID if nsteps < 1 or as mpk_cheb.                */
int mpk_cheb_steps(mpk_plan_t plan, const double *coef, int32_t M, double c, double r, int32_t nsteps,
                   const void *x, double *y, uint32_t flags);

/* mpk_cheb and mpk_cheb_real with x and y in HOST memory (same layouts,
 * coefficients and flags): x is copied to a stream-ordered device buffer,
 * the propagation runs, and y is copied back, all on the plan's stream
 * (page-locked host memory for full-speed copies; pageable is accepted).
 * With MPK_ASYNC, synchronise the plan's stream before reading y.  Errors
 * as the device forms, and MPK_ERR_OOM when the staging buffers cannot be
 * allocated.                                                               */
int mpk_cheb_host(mpk_plan_t plan, const double *coef, int32_t M, double c, double r,
                  const void *x_host, double *y_host, uint32_t flags);
int mpk_cheb_real_host(mpk_plan_t plan, const double *coef, int32_t M, double c, double r,
                       const void *x_host, double *y_host, uint32_t flags);

/* ---------------------------------------------------------------- batches
 * Several plans (different matrices, sizes, block widths nrhs and powers p)
 * run in ONE persistent wavefront launch: their issue orders (each the
 * diagonal order of its own Lp diagram, with the plan's own work-item size,
 * f and sweep length) are merged by relative position, so every plan keeps
 * its dependency order, and the items of all plans share the CTAs of the
 * GPU.  Plans must have the same precision (MPK_F64 or
 * MPK_F32; MPK_F32_BF16VAL is MPK_ERR_UNSUPPORTED) and device, and must not be
 * run on their own while the batch runs (they share their dependency flags).
 * The batch uses the stream of plans[0].  Vectors are in each plan's level
 * order (as with MPK_IO_PERMUTED).                                          */
typedef struct mpk_batch_s *mpk_batch_t;

/* Builds the merged issue order of `count` plans (host array of handles,
 * 1 <= count <= 1024; the batch keeps pointers to the plans, which must
 * outlive it).                                                            */
int mpk_batch_create(const mpk_plan_t *plans, int32_t count, mpk_batch_t *out);

/* Number of work items and CTAs of the batched launch (host outputs).     */
int mpk_batch_info(mpk_batch_t batch, int32_t *n_items, int32_t *grid_ctas);

/* One launch: Ys[m][k-1] = A_m^k xs[m] for every plan m.  xs, Ys: HOST arrays
 * of `count` DEVICE pointers (layouts as for mpk_run).  Errors as mpk_run.  */
int mpk_batch_run(mpk_batch_t batch, const void *const *xs, void *const *Ys, uint32_t flags);

/* Captures the batched launch for these xs / Ys into a CUDA graph (on a
 * private stream) and keeps its executable instance in the batch.          */
int mpk_batch_graph_capture(mpk_batch_t batch, const void *const *xs, void *const *Ys);

/* Replays the captured graph on the batch's stream (MPK_ASYNC: no sync and
 * no error read-back).  MPK_ERR_INVALID if nothing was captured.           */
int mpk_batch_graph_launch(mpk_batch_t batch, uint32_t flags);

/* Releases the batch (not its plans).  NULL is accepted.                   */
int mpk_batch_destroy(mpk_batch_t batch);

/* ---------------------------------------------------------------- tuning
 * The parameters of the method (Sec. 5: the cache budget C of Eq. 5 through
 * f, and how a power k is split into sweeps of p_m powers, Sec. 5.1) plus
 * the GPU work-item size, searched by timing on the GPU.                    */
typedef struct {
    int32_t tile_rows;     /* in: rows per work item (0: automatic)           */
    double safety_f;       /* in: f of Eq. 5 (with the base C)                */
    uint32_t tune;         /* in: MPK_TUNE_* bits                             */
    int32_t p_sweep;       /* in: powers per sweep (mpk_opts.sweep: the k
                              powers in one launch, sweeps of p_sweep; with
                              MPK_TUNE_RESIDENT one plan and launch per sweep
                              of p_sweep powers and one for the rest)         */
    double ms;             /* out: measured time of the k powers (ms), -1 if failed */
    int32_t status;        /* out: mpk_status of planning / running           */
} mpk_tune_candidate;

/* Fills out[0..*count) with the default search grid for k powers: entry 0 is
 * the library's default options (tile_rows 0, f 0.5, p_sweep k); then the
 * resident schedule (MPK_TUNE_RESIDENT, tiles sized to the stage) for p_sweep
 * in {k, ceil(k/2) when k >= 4}; then work items of 64/128/256/512/1024 rows
 * x f in {0.25, 0.5} x p_sweep in {k, ceil(k/2) when k >= 4, 1 when k >= 2}.
 * MPK_ERR_INVALID if max is too small (count = entries written).            */
int mpk_tune_default_grid(int32_t k, mpk_tune_candidate *out, int32_t max, int32_t *count);

/* Times every candidate for the MPK of A with k powers (opts from *base with
 * the candidate's fields; each plan run repeatedly until min_time_s),
 * writes ms / status into cand[], and *best = the index of the fastest.
 * Allocates temporary device vectors.  MPK_ERR_UNSUPPORTED if no candidate
 * ran; MPK_ERR_CUDA ends the search.                                        */
int mpk_autotune(const mpk_csr *A, int32_t k, const mpk_opts *base, double min_time_s, mpk_tune_candidate *cand,
                 int32_t n_cand, int32_t *best);

/* ---------------------------------------------------------------- planner network
 * The multilayer perceptron of the learned planner (no counterpart in the
 * paper; the paper tunes by search, Sec. 6.1): n_in -> n_hidden (ReLU) ->
 * n_hidden (ReLU) -> n_out (linear), FP32, trained on the GPU with a masked
 * mean-squared error sum_ij M_ij (Y_ij - T_ij)^2 / sum_ij M_ij and Adam.
 * Parameters (flat, FP32): W1[n_hidden][n_in], b1, W2[n_hidden][n_hidden],
 * b2, W3[n_out][n_hidden], b3; Glorot-uniform weights from SplitMix64(seed),
 * zero biases.  X, T, M, Y are DEVICE row-major [batch][...] arrays.        */
typedef struct mpk_mlp_s *mpk_mlp_t;

int mpk_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_out, uint64_t seed, void *stream, mpk_mlp_t *out);
/* Number of parameters (or MPK_ERR_INVALID).                               */
int32_t mpk_mlp_num_params(mpk_mlp_t net);
/* Copy parameters to / from HOST memory (count must equal the number of
 * parameters; setting also resets the Adam moments).                      */
int mpk_mlp_get_params(mpk_mlp_t net, float *host, int32_t count);
int mpk_mlp_set_params(mpk_mlp_t net, const float *host, int32_t count);
/* Y[batch][n_out] = net(X[batch][n_in]).                                   */
int mpk_mlp_forward(mpk_mlp_t net, const float *X, int32_t batch, float *Y);
/* Loss (host *loss) and gradient of all parameters for one batch; the
 * gradient stays on the device for mpk_mlp_adam_step and is copied to HOST
 * grad_host[num_params] when that is not NULL.                             */
int mpk_mlp_loss_grad(mpk_mlp_t net, const float *X, const float *T, const float *M, int32_t batch, double *loss,
                      float *grad_host);
/* One Adam update with the last gradient.                                  */
int mpk_mlp_adam_step(mpk_mlp_t net, float lr, float beta1, float beta2, float eps);
int mpk_mlp_destroy(mpk_mlp_t net);

/* ---------------------------------------------------------------- Krylov consumers
 * Solvers of A x = b for a symmetric positive definite A that use the
 * plan's kernels (Sec. 1: s-step Krylov methods get their Krylov basis of s
 * powers from one MPK).  FP64 plans.  b, x: n DEVICE doubles in the caller's
 * numbering (MPK_IO_PERMUTED: the plan's level order); x holds the initial
 * guess on entry and the solution on return.  The iteration stops when the
 * recurred residual satisfies ||r|| <= tol * ||b|| or after max_steps CG
 * steps; *steps and *relres (HOST) receive the steps taken and
 * ||r|| / ||b||.  Work space is plan-owned (allocated on first use).
 * Calls synchronise the plan's stream.  Errors: MPK_ERR_INVALID (NULL
 * pointers, tol < 0, max_steps < 0, a plan of another precision or width),
 * MPK_ERR_OOM, MPK_ERR_CUDA, MPK_ERR_TIMEOUT.                               */

/* Conjugate gradients (Hestenes and Stiefel): one SpMV and two inner
 * products per step, the scalars kept on the device (the residual norm is
 * read back every 8 steps, so up to 7 steps may follow convergence).  Plan:
 * nrhs = 1, MPK_F64.                                                        */
int mpk_cg(mpk_plan_t plan, const double *b, double *x, double tol, int32_t max_steps, int32_t *steps,
           double *relres, uint32_t flags);

/* s-step CG with the monomial basis: per s steps, ONE level-blocked MPK of
 * the block [p r] (the plan: nrhs = 2, MPK_F64, p = s in 1..16) gives
 * V = [p, Ap/rho, .., A^s p/rho^s, r, Ar/rho, .., A^(s-1) r/rho^(s-1)], its
 * Gram matrix V^T V is summed on the GPU (FP64), s CG steps run on the
 * coefficient vectors of the 2s+1 columns (with ||r||^2 from the Gram
 * matrix), and one fused pass forms x, p and r.  rho scales the basis
 * (0 = the larger end of the Gershgorin interval); the monomial basis loses
 * accuracy as s grows, so s of 4..8 with rho near ||A|| is the usual choice. */
int mpk_sstep_cg(mpk_plan_t plan, const double *b, double *x, double tol, int32_t max_steps, double rho,
                 int32_t *steps, double *relres, uint32_t flags);

/* Reorders vectors between the caller's numbering and the plan's level
 * order (Sec. 4.5: the permutation vector recovers the original order).
 * src and dst: count blocks of n x nrhs elements of elem_bytes (4 or 8)
 * each, not overlapping.  to_level != 0: dst[r] = src[perm[r]]; else
 * dst[perm[r]] = src[r].                                                   */
int mpk_permute_vectors(mpk_plan_t plan, const void *src, void *dst, int32_t count,
                        int32_t elem_bytes, int32_t to_level);

/* Releases the plan and all its device memory (after finishing its stream's
 * work).  NULL is accepted.                                                */
int mpk_plan_destroy(mpk_plan_t plan);

/* Test hook for the bounded waits: the NEXT wavefront launch of this plan
 * does not publish the completion of work item (tile, power), so the items
 * that read it reach their wait limit (opts.timeout_s) and the call returns
 * MPK_ERR_TIMEOUT with that node in mpk_plan_last_error; later launches are
 * unaffected.  No fault, trap or unbounded wait is involved.  tile < 0
 * cancels a pending drop.  MPK_ERR_INVALID for an item outside the plan.  */
int mpk_plan_debug_drop_flag(mpk_plan_t plan, int32_t tile, int32_t power);

/* Levels of Eq. 3 (the same values as mpk_plan_perm's level[] for a plan
 * built with assume_symmetric != 0 and the same root) WITHOUT ANY DEVICE
 * ALLOCATION.  The paper has no counterpart: this entry point exists for
 * callers that must not allocate device memory, for example a host that
 * sizes all device memory at start-up and forbids allocation afterwards
 * (an embedded service under a fixed memory budget, or a process that
 * shares the GPU under a hard quota).  mpk_plan allocates, so such callers
 * use this call.
 *
 * The scratch (frontier queue and control words) is a static device array
 * inside this library, sized for n <= 1,048,576 vertices (about 4 MB, held
 * on every GPU that loads the library until the process exits).  The caller
 * passes the inputs and the output: n, nnz and the CRS arrays rowptr[n+1],
 * col[nnz] (DEVICE, caller-owned; the stored pattern is taken as symmetric),
 * the root, and level[n] (DEVICE, caller-allocated, overwritten).  *n_levels
 * (host) receives L_m.  stream: cudaStream_t; timeout_s bounds each wait of
 * the kernel (0 = 2 s).
 *
 * The call synchronises the stream twice and reads a status word back to the
 * host (the validation result and the level count), so it must not be
 * issued on a stream that is being captured into a CUDA graph.  Each call
 * looks up the device address of the array in the current device's context
 * (which may load the library's device code on the first call).  Every call
 * shares the one array and clears its control words on entry: calls that
 * overlap on the GPU (other streams, other host threads) race and must not
 * be issued.
 *
 * Errors: MPK_ERR_UNSUPPORTED if n > 1,048,576 (the scratch limit);
 * MPK_ERR_INVALID for NULL pointers, n < 1, a root outside [0, n) or a
 * malformed CRS (found on the device); MPK_ERR_TIMEOUT, MPK_ERR_CUDA.      */
int mpk_levels_noalloc(int32_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col, int32_t root,
                       int32_t *level, int32_t *n_levels, void *stream, double timeout_s);

/* Arithmetic-rate probe for an ALU roofline (the paper measures its
 * machine's limits with microbenchmarks too, Sec. 2): launches, on `stream`
 * (cudaStream_t) and without waiting, SMs x blocks_per_sm CTAs of 256
 * threads, each thread running 8 independent chains of `iters` dependent
 * fused multiply-adds in FP64 (prec = MPK_F64) or FP32 (prec = MPK_F32).
 * *flops (host) receives the flops of the launch (2 per FMA); the caller
 * times the launch (CUDA events on the same stream) for the rate.  sink:
 * DEVICE buffer of at least 8 bytes (never written in practice; it keeps
 * the chains live).  MPK_ERR_INVALID for a NULL pointer, another prec,
 * blocks_per_sm outside [1, 32], or iters not a positive multiple of 4.     */
int mpk_probe_fma(int32_t prec, int32_t blocks_per_sm, int64_t iters, void *sink, void *stream, double *flops);

/* Static description of a status code.                                     */
const char *mpk_strerror(int status);

/* Detail of the last device-side error of the plan (host outputs; any may be
 * NULL): code (an mpk_status), the power k and the work item (tile) whose
 * wait expired.                                                            */
int mpk_plan_last_error(mpk_plan_t plan, int32_t *code, int32_t *power, int32_t *tile);

#ifdef __cplusplus
}
#endif
#endif /* MPK_H */
