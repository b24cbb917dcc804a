/*
 * iluk.h -- C ABI of libiluk: ILU(k) preconditioning for sparse non-symmetric
 * Ax = b on one NVIDIA GB300 (sm_103a), after Dong & Cooperman, "A
 * Bit-Compatible Shared Memory Parallelization for ILU(k) Preconditioning and
 * a Bit-Compatible Generalization to Distributed Memory" (arXiv 0803.0048).
 *
 * The calls follow the paper's statement of the problem (Sec. 2): a symbolic
 * phase that fixes the level-k pattern, a numeric phase that fills in the
 * values of the incomplete factors, a triangular solve L~U~y = p applied in
 * every iteration of a Krylov solver, and, as an option, the level-based
 * incomplete inverse (TPIILU, Sec. 3.5) that turns that solve into two sparse
 * mat-vecs.
 *
 * The steps are numbered the same way here and in the library's sources:
 *   a1 pattern check            a5 TPIILU build and apply
 *   a2 symbolic phase           a6 restarted GMRES(m)
 *   a3 numeric phase            a7 many systems on one pattern (batched)
 *   a4 triangular sweeps        a8 gradient of a solve (adjoint)
 *
 * General conventions (all entry points):
 *  - Matrices are CSR, 0-based: rowptr int64[n+1] (rowptr[0] = 0,
 *    non-decreasing), colind int32[nnz] strictly ascending inside each row,
 *    values double[nnz].  An entry stored in the CSR arrays counts as
 *    structurally non-zero whatever its value.
 *  - Pointers named in these signatures are DEVICE pointers unless the
 *    comment says "host".  They are borrowed for the duration of the call (or,
 *    for asynchronous calls, until the stream reaches the work).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  All device work of a call is ordered on that stream.
 *  - Handles (iluk_sym, iluk_fac, iiluk) own the device memory they allocate
 *    (stream-ordered cudaMallocAsync on the creating call's stream) until the
 *    matching *_destroy.  A handle must not be used concurrently from two
 *    streams: the sweeps keep per-handle scratch (flags, an intermediate
 *    vector) inside it.
 *  - Return value: an iluk_status.  Calls documented as "synchronous"
 *    synchronize `stream` before returning and also fill `info` (may be NULL).
 *    Calls documented as "asynchronous" only enqueue work; device-side errors
 *    they meet (a bounded wait that gave up) are recorded in the handle and
 *    returned by the next synchronous call on it, or by iluk_fac_status().
 *  - No call traps or aborts the GPU on bad input: every device-side check
 *    records a status and the kernels return.  Every wait of one row on
 *    another is bounded (iluk_set_wait_limit); running out returns
 *    ILUK_ETIMEOUT.
 *  - Floating point: every kernel computes in IEEE double with one rounding
 *    per multiply and per add (no fused multiply-add) and correctly rounded
 *    division and square root, in the sequential per-entry order of the
 *    method, so the results are bit-identical to a sequential run.
 */
#ifndef ILUK_H
#define ILUK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ILUK_OK = 0,
  ILUK_EINVAL = 1,      /* bad argument (n < 0, k out of range, NULL pointer, ...)      */
  ILUK_EPATTERN = 2,    /* unsorted / duplicate / out-of-range column, bad rowptr       */
  ILUK_ENODIAG = 3,     /* a row has no diagonal entry after the symbolic phase         */
  ILUK_EZEROPIVOT = 4,  /* a diagonal u_ii of the factors is exactly 0.0                */
  ILUK_ENONFINITE = 5,  /* a matrix value is NaN or infinite                            */
  ILUK_ENOMEM = 6,      /* device allocation failed or a row exceeds the supported size */
  ILUK_ETIMEOUT = 7,    /* a bounded wait on another row's completion gave up           */
  ILUK_ENOCONV = 8,     /* GMRES reached maxit without meeting rtol                     */
  ILUK_ECUDA = 9        /* a CUDA runtime call failed                                   */
} iluk_status;

/* Sparsity pattern of A (device arrays). */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int64_t *rowptr;  /* int64[n+1] */
  const int32_t *colind;  /* int32[nnz] */
} iluk_pattern;

/* Result details of a synchronous call. */
typedef struct {
  int32_t status;   /* same as the return value                                    */
  int32_t iters;    /* GMRES: Arnoldi steps taken                                  */
  int64_t row;      /* first failing row (sequential order), or -1                 */
  double relres;    /* GMRES: true ||b - Ax|| / ||b|| at exit                      */
  int64_t need;     /* ILUK_ENOMEM: bytes or entries that were needed (if known)   */
  int32_t cycles;   /* GMRES: restart cycles started                               */
  int32_t reserved;
} iluk_info;

/* Read-only view of a symbolic result (device pointers borrowed from S). */
typedef struct {
  int64_t n;
  int64_t nnz;              /* entries of F = L~ + U~ (diagonal in U~)              */
  const int64_t *rowptr;    /* int64[n+1]                                          */
  const int32_t *colind;    /* int32[nnz], sorted within rows                       */
  const uint8_t *level;     /* uint8[nnz], level of fill of each entry (Def. 2.3)   */
  const int64_t *diag;      /* int64[n], position of (i,i) in colind                */
  const int32_t *a2f;       /* int32[nnz_A], offset of A's entry inside its F row   */
  int32_t max_row;          /* longest row of F                                    */
  int32_t depth_lower;      /* longest dependency chain of the forward sweep, or -1 */
  int32_t depth_upper;      /* ... of the backward sweep, or -1: both are -1 until
                               the level orders exist (first iluk_numeric on S, or
                               iluk_sym_depth)                                      */
  int32_t k;
} iluk_sym_view;

typedef struct iluk_sym iluk_sym;  /* symbolic result: pattern of F and levels */
typedef struct iluk_fac iluk_fac;  /* numeric factors L~, U~ on that pattern   */
typedef struct iiluk iiluk;        /* TPIILU incomplete inverses              */

enum { ILUK_PREC_NONE = 0, ILUK_PREC_ILU = 1, ILUK_PREC_IILU = 2 };
/* Sweep schedules (all give bit-identical results): rows of a level in
 * lockstep warps over all SMs (FLAGS), on one SM (SINGLE_CTA) or on one
 * thread-block cluster (CLUSTER); one warp per row over all SMs (WARP_GRID)
 * or on one cluster (WARP_CLUSTER).  AUTO times them and keeps the fastest;
 * the pick is remembered by the symbolic handle, and later factorizations of
 * the same pattern use it without timing again.
 * A schedule byte holds the kind in bits 0-3 and, for the warp-per-row
 * kinds, the threads per CTA / 128 in bits 4-7 (0: 1024 threads; for
 * WARP_GRID a non-zero width also means one CTA per SM), which bounds how
 * many rows are in flight: ILUK_SCHED_WIDTH(ILUK_SCHED_WARP_CLUSTER, 512). */
/* WARP_CLUSTER_HELP is WARP_CLUSTER plus a second 16-CTA cluster of prefix
 * helpers in the same cooperative launch: for each row, shortly before its
 * warp takes it, a helper warp on another SM subtracts the products of the
 * row's leading entries whose x is already final and hands the partial
 * difference over, so most of each subtraction chain runs off the SMs of the
 * critical path (same operations in the same order: same bits).  It keeps
 * per-row scratch in F (16 bytes a row) and runs as WARP_CLUSTER when the
 * GPU cannot hold both clusters at once.  Widths as for WARP_CLUSTER. */
enum {
  ILUK_SCHED_AUTO = 0, ILUK_SCHED_FLAGS = 1, ILUK_SCHED_SINGLE_CTA = 2, ILUK_SCHED_CLUSTER = 3,
  ILUK_SCHED_WARP_GRID = 4, ILUK_SCHED_WARP_CLUSTER = 5, ILUK_SCHED_WARP_CLUSTER_HELP = 6
};
#define ILUK_SCHED_WIDTH(kind, threads) ((kind) | (((threads) / 128) << 4))

const char *iluk_strerror(int status);

/* Upper bound, in nanoseconds, on any single wait of a row for another row's
 * completion inside the kernels (default 20 s).  Host-side setting for the
 * whole process; returns the previous value. */
int64_t iluk_set_wait_limit(int64_t ns);

/* Test hook for the bounded-wait path: the factorization row `row` (-1 = none)
 * finishes its work but never publishes its completion, so every row that
 * depends on it runs out its wait and the call returns ILUK_ETIMEOUT.  Returns
 * the previous value.  Host-side, whole process. */
int64_t iluk_debug_hold_row(int64_t row);

/* The symbolic phase for k <= 1, where rows need no other row's pattern
 * (Sec. 3.3): 0 (default) each warp takes the next row in ascending order and
 * reads its pivot rows from A without waiting; 1 the same, last row first
 * (the order Sec. 3.3 found fastest on a CPU); 2 the general walk of k >= 2
 * (rows announce their arena slots and dependants wait for them).  All three
 * give the same pattern and levels; the setting exists to compare them.
 * Host-side, whole process; returns the previous variant, or -1 (and changes
 * nothing) for an unknown one. */
int iluk_set_symbolic_variant(int variant);

/* Number of CUDA kernels this library has launched in the process so far
 * (memsets and copies are not counted). */
int64_t iluk_launch_count(void);

/* Kernel timing.  While enabled, every kernel launch of the kinds below is
 * bracketed by CUDA events on its own stream.  iluk_prof_read synchronizes
 * those events and fills ms[kind] (total milliseconds) and count[kind]
 * (launches) for kind < nkinds (host arrays).  Enabling clears the records.
 * OVERLAPPED collects the work a call runs on a second stream beside its main
 * kernel (the level orders built during the first numeric phase of a
 * pattern): its time is hidden, not added, so it is kept apart. */
enum {
  ILUK_PROF_VALIDATE = 0, ILUK_PROF_SYMBOLIC = 1, ILUK_PROF_COMPACT = 2, ILUK_PROF_DEPTH = 3,
  ILUK_PROF_NUMERIC = 4, ILUK_PROF_SWEEP = 5 /* forward sweeps */, ILUK_PROF_TRANSPOSE = 6, ILUK_PROF_IILU_BUILD = 7,
  ILUK_PROF_IILU_APPLY = 8, ILUK_PROF_SPMV = 9, ILUK_PROF_DOT = 10, ILUK_PROF_VECTOR = 11,
  ILUK_PROF_SWEEP_BWD = 12, ILUK_PROF_BATCH = 13, ILUK_PROF_OVERLAPPED = 14,
  ILUK_PROF_FACTOR = 15 /* symbolic and numeric in one launch (iluk_factor) */, ILUK_PROF_KINDS = 16
};
int iluk_prof_enable(int on);
int iluk_prof_read(double *ms, int64_t *count, int nkinds);

/*
 * a1. Pattern check (sparse storage, Sec. 2.1).  Synchronous.
 * Checks rowptr[0] = 0, rowptr non-decreasing, rowptr[n] = nnz, every column in
 * [0, n) and strictly ascending inside its row.  ILUK_EPATTERN with the
 * smallest failing row in info->row.
 */
int iluk_validate(const iluk_pattern *A, iluk_info *info, void *stream);

/*
 * a2. Symbolic factorization, Phase I (Algorithm 1, Sec. 2.2) with the level
 * of fill of Def. 2.3: level(i,j) = 0 for stored a_ij, otherwise
 * min_{h < min(i,j)} level(i,h) + level(h,j) + 1; entries of level <= k are
 * kept.  0 <= k <= 250.  Synchronous.  Validates A first (as iluk_validate).
 * On success *S receives a new handle holding F's pattern, the levels, the
 * diagonal positions and the A->F position map.  ILUK_ENODIAG (row in
 * info->row) when some row of F lacks its diagonal.  A is only read; it may be
 * freed after the call.
 */
int iluk_symbolic(const iluk_pattern *A, int k, iluk_sym **S, iluk_info *info, void *stream);
int iluk_sym_query(const iluk_sym *S, iluk_sym_view *view);
/* Longest dependency chains of the forward and backward sweeps over F's
 * pattern (the number of rows on the critical path of each sweep).  They come
 * with the sweeps' level orders, which the first iluk_numeric on S builds on a
 * second stream while it factorizes; if none has run yet, this call builds
 * them (synchronous on `stream`).  Cached in S afterwards. */
int iluk_sym_depth(iluk_sym *S, int32_t *depth_lower, int32_t *depth_upper, void *stream);
/* Copy S's arrays into caller-owned device buffers (any pointer may be NULL
 * to skip that array).  Asynchronous. */
int iluk_sym_export(const iluk_sym *S, int64_t *rowptr, int32_t *colind, uint8_t *level,
                    int64_t *diag, void *stream);
void iluk_sym_destroy(iluk_sym *S);

/*
 * a3. Numeric factorization, Phase II, row-wise IKJ elimination (Eq. 1;
 * Eqs. lufactor2, lufactor of Sec. 3.5): F starts as A on F's pattern (fill
 * positions +0.0); for each row i and each h in L(i) ascending,
 * f_ih <- f_ih / f_hh, then f_ij <- f_ij - f_ih * f_hj for every j > h stored
 * in both rows.  A_val: device double[nnz_A] in S's A pattern order.
 * Synchronous.  *F receives a new handle (it refers to S, which must outlive
 * it).  ILUK_EZEROPIVOT / ILUK_ENONFINITE with the first failing row.
 */
int iluk_numeric(const iluk_sym *S, const double *A_val, iluk_fac **F, iluk_info *info,
                 void *stream);
/* Re-run the numeric phase into an existing handle with new values. */
int iluk_refactor(iluk_fac *F, const double *A_val, iluk_info *info, void *stream);
/*
 * a2 + a3 together: iluk_symbolic(A, k) then iluk_numeric, with the numeric
 * phase running beside the symbolic one (k >= 2: one launch in which each row
 * is factored as soon as its pattern is final, its values kept in an arena
 * laid out like the symbolic one until both phases end).  *S and *F receive
 * handles equal, bit for bit, to those of the two calls, except that the
 * level orders of the sweeps are not built: the sweeps walk rows in index
 * order (ascending forward, descending backward; any order that puts every
 * dependency first gives the same bits) until a later iluk_numeric or
 * iluk_refactor on S, or iluk_sym_depth, builds them (on wide DAGs, such as 3D
 * grids, level orders give much faster sweeps: call iluk_sym_depth first, or
 * the two calls).  For k <= 1 the two phases run one after the other (rows
 * need no other rows' patterns), also without level orders.  Falls back to the
 * two calls for rows of F longer than 512 entries and whenever the combined
 * launch reports an error (the two calls then report it).
 * Synchronous; errors as iluk_symbolic and iluk_numeric.
 */
int iluk_factor(const iluk_pattern *A, const double *A_val, int k, iluk_sym **S, iluk_fac **F,
                iluk_info *info, void *stream);
/* Device pointer to the factor values (double[nnz_F], F's pattern order). */
int iluk_fac_values(const iluk_fac *F, const double **val);
/* Copy the factor values into a caller-owned device buffer double[nnz_F].
 * Asynchronous. */
int iluk_fac_export(const iluk_fac *F, double *val, void *stream);
/* Status recorded by asynchronous calls on F since the last query; clears it. */
int iluk_fac_status(iluk_fac *F, iluk_info *info, void *stream);
void iluk_fac_destroy(iluk_fac *F);

/*
 * a4. Preconditioner application (Eq. triangleSolve): y = (L~U~)^-1 p by a
 * forward sweep x_i = p_i - sum_{h<i} f_ih x_h (Eq. forwardsubA, h ascending)
 * and a backward sweep y_i = (x_i - sum_{j>i} f_ij y_j) / f_ii (j descending:
 * each row read right to left, the mirror image of the forward sweep).
 * With transpose != 0: y = (L~U~)^-T p = L~^-T U~^-T p on the explicit
 * transpose of F (built on the first transposed call; make that first call
 * outside any stream capture).  p, y: device double[n]; p and y may alias.
 * Asynchronous.  `sched` picks the schedule (ILUK_SCHED_*).
 */
int iluk_apply(iluk_fac *F, const double *p, double *y, int transpose, void *stream);
int iluk_apply_sched(iluk_fac *F, const double *p, double *y, int transpose, int sched,
                     void *stream);
/* Fix the sweep schedule of F: one schedule byte for both sweeps, or
 * forward | backward << 8; it applies to the sweeps of F and of its
 * transpose.  ILUK_SCHED_AUTO (the default) lets the first application
 * outside a stream capture time every schedule (and, for the warp-per-row
 * kinds, several CTA widths) on each sweep and keep the fastest
 * (iluk_get_schedule then returns the packed pair); the transposed sweeps are
 * timed on their first use and keep their own pair.  Both picks are
 * remembered by the symbolic handle: later factorizations of the same
 * pattern use them without timing again.  An unknown kind or width is
 * refused (ILUK_EINVAL). */
int iluk_set_schedule(iluk_fac *F, int sched);
int iluk_get_schedule(const iluk_fac *F);

/*
 * a5. TPIILU (Sec. 3.5).  Build: beta_it = f_it - sum_{t<h<i} f_ih beta_ht on
 * F's lower pattern (Eq. inversedefine, h ascending), and the mirror image
 * gamma_it = u^_it - sum_{i<h<t} u^_ih gamma_ht with u^_it = u_it / u_ii on the
 * strictly upper pattern (rows last to first, h descending).  The result g is
 * aligned with F: -beta on lower positions, -gamma on strictly upper positions,
 * u_ii on the diagonal.  Synchronous; *M receives a new handle that refers to
 * F's symbolic handle.
 * Apply: y = (I + G_U) D^-1 (I + G_L) p, each row summed left to right with the
 * own term added last.  Asynchronous.
 */
int iiluk_build(const iluk_fac *F, iiluk **M, iluk_info *info, void *stream);
int iiluk_values(const iiluk *M, const double **g);
/* Copy g into a caller-owned device buffer double[nnz_F].  Asynchronous. */
int iiluk_export(const iiluk *M, double *g, void *stream);
int iiluk_apply(const iiluk *M, const double *p, double *y, void *stream);

/*
 * The same TPIILU apply for callers that cannot allocate device memory (their
 * memory belongs to another runtime or a fixed pool, or allocation is not
 * allowed where they run).  Not from the paper, which has no counterpart: an
 * interface addition.  The caller passes F's pattern (rowptr int64[n+1],
 * colind int32[nnz], diag int64[n], as exported by iluk_sym_export), the
 * TPIILU values g (double[nnz], as exported by iiluk_export), p and y (device
 * double[n]); the result is bit-identical to iiluk_apply.  The intermediate
 * vector lives in a static device array of ILUK_NOALLOC_MAX_N doubles (8 MiB)
 * that every device loading the library keeps until exit; n above that limit
 * returns ILUK_ENOMEM.  The call allocates nothing.  The first call on a
 * device looks up the array's device address (make it before any stream
 * capture).  All calls share the one array: calls that overlap on the GPU
 * (other streams, or other host threads) race on it.  Asynchronous.
 */
#define ILUK_NOALLOC_MAX_N (1 << 20)
int iiluk_apply_noalloc(int64_t n, const int64_t *rowptr, const int32_t *colind,
                        const int64_t *diag, const double *g, const double *p, double *y,
                        void *stream);
void iiluk_destroy(iiluk *M);

/*
 * Sparse mat-vec y = A x (transpose = 0; each row summed left to right from
 * +0.0) on A's pattern and values.  Asynchronous.
 */
int iluk_spmv(const iluk_pattern *A, const double *A_val, const double *x, double *y,
              void *stream);

/*
 * Fixed-order inner product: 4096 partial sums, partial p summing i = p,
 * p+4096, ... left to right from +0.0, then the pairwise tree
 * s[p] += s[p+w] for w = 2048, ..., 1.  out: device double[1].  Asynchronous.
 */
int iluk_dot(int64_t n, const double *x, const double *y, double *out, void *stream);

/*
 * Elementwise q_i = a_i / b_i rounded to nearest, computed as the numeric
 * phase forms its multipliers f_ih / f_hh (Eq. lufactor2) and as the sweeps
 * divide by u_ii (Eq. triangleSolve): on the integer pipes, from a 64-bit
 * fixed-point reciprocal of b_i (an fp32 seed refined by two Newton steps)
 * and an exact remainder correction, with IEEE division for zero, subnormal,
 * infinite and NaN operands and for quotients outside the normal range.  The
 * results must equal IEEE division bit for bit; this call exists so that the
 * method can be checked against it.  a, b, q: device double[n] (q may alias
 * neither).  ILUK_EINVAL on n < 0 or a null pointer with n > 0.  Asynchronous.
 */
int iluk_div_rn(int64_t n, const double *a, const double *b, double *q, void *stream);

/*
 * a6. Restarted GMRES(m), right preconditioned (the solver works with
 * A M^-1, Sec. 2), x0 = 0, modified Gram-Schmidt with the fixed-order inner
 * product above, Givens rotations.  Stops when |g_{j+1}| / ||b|| <= rtol and
 * the true residual ||b - Ax|| / ||b|| confirms it at the end of the cycle.
 * prec_kind: ILUK_PREC_NONE (prec ignored), ILUK_PREC_ILU (prec = iluk_fac*),
 * ILUK_PREC_IILU (prec = iiluk*).  transpose != 0 solves A^T x = b with
 * M^-T (ILU only).  b, x: device double[n].  maxit bounds the total number of
 * Arnoldi steps.  Synchronous; ILUK_ENOCONV when maxit is reached.
 */
int gmres_solve(const iluk_pattern *A, const double *A_val, int prec_kind, void *prec,
                const double *b, double *x, int restart, double rtol, int maxit,
                int transpose, iluk_info *info, void *stream);

/*
 * a6, a8. The same GMRES(m) with a choice of what a restart cycle keeps for
 * its final update (the memory of the Krylov bases).  gmres_solve is
 * gmres_solve_ex with ILUK_BASIS_AUTO.
 *  ILUK_BASIS_STORE      keeps the preconditioned basis z_j = M^-1 v_j
 *                        (m more vectors of n doubles) and ends a cycle with
 *                        x += Z y (the flexible form, Saad 1993).
 *  ILUK_BASIS_RECOMPUTE  keeps only V and, at the end of a cycle, applies M to
 *                        each v_j again and accumulates Z y term by term in
 *                        the same order: bit-identical to STORE, at the cost
 *                        of up to m more applications of M per cycle.
 *  ILUK_BASIS_AUTO       STORE when the m vectors take at most half of the
 *                        device's free memory, else RECOMPUTE (same bits).
 *  ILUK_BASIS_MINV_VY    keeps only V and ends a cycle with x += M^-1 (V y),
 *                        the textbook form of right preconditioning (Sec. 2's
 *                        A U~^-1 L~^-1): one more application of M per cycle;
 *                        equal to the forms above in exact arithmetic, not in
 *                        rounding.
 * Other arguments, results and errors as gmres_solve (ILUK_EINVAL for an
 * unknown basis).  Synchronous.
 */
enum { ILUK_BASIS_AUTO = 0, ILUK_BASIS_STORE = 1, ILUK_BASIS_RECOMPUTE = 2,
       ILUK_BASIS_MINV_VY = 3 };
int gmres_solve_ex(const iluk_pattern *A, const double *A_val, int prec_kind, void *prec,
                   const double *b, double *x, int restart, double rtol, int maxit,
                   int transpose, int basis, iluk_info *info, void *stream);

/*
 * Preconditioned BiCGSTAB (van der Vorst 1992), the solver of the paper's
 * experiments (Sec. 4), right preconditioned, x0 = 0, shadow residual r^ = b,
 * inner products in the fixed order above.  Per iteration, each operation
 * rounded once: rho = (r^,r); p = r + beta (p - omega v) with beta =
 * (rho/rho_prev)(alpha/omega) (p = r first); p^ = M^-1 p; v = A p^;
 * alpha = rho / (r^,v); s = r - alpha v; stop with x += alpha p^ when
 * ||s||/||b|| <= rtol; s^ = M^-1 s; t = A s^; omega = (t,s)/(t,t);
 * x = (x + alpha p^) + omega s^; r = s - omega t; stop when ||r||/||b|| <= rtol.
 * info->relres is the true ||b - Ax||/||b|| at exit, info->iters the
 * iterations.  prec_kind / prec as for gmres_solve (no transpose).  b, x:
 * device double[n].  Synchronous; ILUK_ENOCONV when maxit is reached,
 * ILUK_EINVAL on a breakdown (rho, (r^,v), (t,t) or omega exactly zero).
 */
int bicgstab_solve(const iluk_pattern *A, const double *A_val, int prec_kind, void *prec,
                   const double *b, double *x, double rtol, int maxit, iluk_info *info,
                   void *stream);

/*
 * The TPILU(k) solve policy (Sec. 1): first the level-based incomplete
 * inverse, and when that does not converge fast, revert to the stable ILU(k)
 * sweeps.  Runs `solver` (ILUK_SOLVER_GMRES with restart `m`, or
 * ILUK_SOLVER_BICGSTAB) preconditioned by M = TPIILU(F) (built and freed here
 * when M is null) for at most iilu_maxit iterations; if that solve does not
 * reach rtol (or breaks down), solves again from x0 = 0 preconditioned by F's
 * sweeps for at most maxit iterations.  *used receives ILUK_PREC_IILU or
 * ILUK_PREC_ILU, the preconditioner of the returned x; info describes that
 * last solve.  Synchronous.
 */
enum { ILUK_SOLVER_GMRES = 0, ILUK_SOLVER_BICGSTAB = 1 };
int tpilu_solve(const iluk_pattern *A, const double *A_val, iluk_fac *F, iiluk *M, int solver,
                const double *b, double *x, int m, double rtol, int iilu_maxit, int maxit,
                int *used, iluk_info *info, void *stream);

/*
 * Explicit CSR transpose: t_rowptr (int64[n+1]), t_colind (int32[nnz]) and
 * t_val (double[nnz]) receive A^T, columns ascending inside each row, values
 * moved exactly.  The transposed solves build the same transposes internally
 * (for A^T lambda = g, and of F for the (L~U~)^-T sweeps); this call gives
 * them to a caller, e.g. to factor A^T on its own.  Caller-owned device
 * buffers; A is not validated.  Asynchronous.
 */
int iluk_transpose(const iluk_pattern *A, const double *A_val, int64_t *t_rowptr,
                   int32_t *t_colind, double *t_val, void *stream);

/*
 * iluk_factor(k) followed by gmres_solve(m, rtol, maxit) preconditioned by
 * the factors, in one call and with the same results bit for bit (x,
 * iterations, cycles, relres; x0 = 0, basis ILUK_BASIS_AUTO), device buffers
 * as those calls take them.  What the one call adds is overlap: the first
 * GMRES vector v_1 = b / ||b|| does not depend on the factors, so it is
 * formed first and the one-launch factorization (k >= 2) solves L x = v_1
 * beside its numeric phase, each row's entry of x computed by the warp that
 * has just factored the row (the forward substitution of Eq. forwardsubA, in the
 * same order and roundings as the forward sweep); the first application of
 * the preconditioner then runs only its backward sweep.  When the one-launch
 * path is not taken (k <= 1, a fallback to the two separate phases) the first
 * application runs both sweeps, as gmres_solve does.  sched is the sweep
 * schedule (as iluk_set_schedule; ILUK_SCHED_AUTO times them once F exists).
 * The factorization is returned through S_out and F_out when both are
 * non-NULL (the caller destroys them), else freed.  A failure of the
 * factorization is reported as iluk_factor reports it (x then holds 0 or is
 * unwritten); the factorization runs even when GMRES needs no iteration.
 * Synchronous.
 */
int iluk_solve(const iluk_pattern *A, const double *A_val, int k, const double *b, double *x,
               int m, double rtol, int maxit, int sched, iluk_sym **S_out, iluk_fac **F_out,
               iluk_info *info, void *stream);

/*
 * a1-a6 in one call, from HOST buffers: rowptr (int64[n+1]), colind
 * (int32[nnz]), val (double[nnz]) and b (double[n]) are host arrays (pinned
 * memory lets the copies run at full speed; pageable memory works too), x
 * (double[n]) is a host array that receives the solution.  The call copies
 * the inputs to the device on `stream`, runs iluk_solve(k, restart, rtol,
 * maxit, sched) on them (iluk_factor(k) and gmres_solve preconditioned by the
 * ILU(k) sweeps, the first forward sweep inside the factorization; with
 * ILUK_SCHED_AUTO the schedules are timed inside the call), copies x back
 * and frees its device memory.
 * Synchronous; statuses and info as the calls it makes (x is written even
 * when GMRES returns ILUK_ENOCONV).
 */
int iluk_solve_host(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *colind,
                    const double *val, const double *b, double *x, int k, int restart,
                    double rtol, int maxit, int sched, iluk_info *info, void *stream);

/*
 * a8 helper. Gradient of a loss through x = A^-1 b with respect to the stored
 * entries of A: gA[p] = -lambda_i * x_j for entry p = (i, j), where lambda
 * solves A^T lambda = dL/dx.  Asynchronous.
 */
int iluk_adjoint_scatter(const iluk_pattern *A, const double *lambda, const double *x,
                         double *gA, void *stream);

/*
 * a7. Batched numeric factorization: nbatch value sets on one pattern.
 * A_vals: device double[nbatch * nnz_A] (set-major); F_vals: device
 * double[nbatch * nnz_F].  One persistent launch.  Every set's factors are
 * bit-identical to iluk_numeric on that set.  infos: host iluk_info[nbatch]
 * (may be NULL).  Synchronous; returns the first failing set's status.
 */
int iluk_numeric_batched(const iluk_sym *S, int64_t nbatch, const double *A_vals,
                         double *F_vals, iluk_info *infos, void *stream);

/*
 * a7. Batched solve: every item is numerically factored (ILU(k) on its
 * symbolic handle) and solved by right-preconditioned GMRES(restart) with the
 * ILU sweeps, all items in ONE persistent launch (each CTA takes the next item
 * and runs its whole pipeline).  Items may have different patterns and sizes;
 * items sharing an iluk_sym share its pattern arrays.  Every item's x (and its
 * iteration count and residual) is bit-identical to iluk_numeric + gmres_solve
 * on that item alone.
 *
 * iluk_batch_create: synchronous; copies the item descriptors (device
 * pointers, borrowed until iluk_batch_destroy) and allocates the workspace.
 * restart <= 64.  The CTAs take the items largest first (by nnz_F + nnz_A +
 * 4 n, ties in item order), so that no large item starts last; results are
 * still reported per item in the caller's order.
 * iluk_batch_solve: asynchronous, no host round trip and no allocation, so it
 * can be recorded in a CUDA graph by stream capture; the first call outside a
 * capture times the CTA widths (256, 512 and 1024 threads per item) and keeps
 * the fastest (autotuner).  New values written into the same a_val / b buffers
 * are picked up by the next call.
 * iluk_batch_results: synchronous; infos (host, may be NULL) gets one entry per
 * item; returns the first item's non-OK status, if any.
 */
typedef struct {
  const iluk_sym *S;        /* symbolic handle of this item's pattern            */
  const int64_t *a_rowptr;  /* device int64[n+1], the pattern S was built from   */
  const int32_t *a_colind;  /* device int32[nnz_A]                               */
  const double *a_val;      /* device double[nnz_A]                              */
  const double *b;          /* device double[n]                                  */
  double *x;                /* device double[n], output                          */
} iluk_batch_item;
typedef struct iluk_batch iluk_batch;

int iluk_batch_create(const iluk_batch_item *items, int64_t nitems, int restart, double rtol,
                      int maxit, iluk_batch **B, void *stream);
int iluk_batch_solve(iluk_batch *B, void *stream);
int iluk_batch_results(iluk_batch *B, iluk_info *infos, void *stream);
/* The first solve outside a stream capture times the whole batch at 256,
 * 512 and 1024 threads per item (as many items at once as fit on each SM:
 * up to four, two, one), each with level-barrier sweeps (every level of the
 * in-CTA sweeps ends at a barrier) and with spinning sweeps (each warp polls
 * the values its rows need, no barriers), and keeps the fastest; the results
 * do not depend on the choice.  Threads per item chosen (0 until the first
 * solve) and whether the sweeps spin (1) or use level barriers (0). */
int iluk_batch_width(const iluk_batch *B);
int iluk_batch_spin(const iluk_batch *B);
/* Fix the schedule instead (width 256, 512 or 1024; ILUK_EINVAL otherwise). */
int iluk_batch_set_schedule(iluk_batch *B, int width, int spin);
void iluk_batch_destroy(iluk_batch *B);

#ifdef __cplusplus
}
#endif
#endif /* ILUK_H */
