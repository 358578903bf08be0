/*
 * sdsl.h -- C ABI of the GB300 (sm_103a) implementation of the SDSL-Solver
 * hot path (arXiv 2604.23979): the preconditioned Krylov solve of the sparse
 * linear systems of an interior-point method.
 *
 * The problem statement is the paper's: one linear system A x = b per
 * interior-point iteration (Algorithm 1), given either in normal-equations
 * form S = B D^{-1} B^T (Eq. schur; here S = A diag(theta) A^T + rho I with
 * theta = the IPM scaling D^{-1}) or in augmented form (Eq. augmented; here
 * K = [[-diag(1/theta), A^T], [A, rho I]]).  The scaling changes every
 * iteration (Sec. 3.4), which is what sdsl_update_diag models.
 *
 * Two parallel methods (Sec. 2.3, 2.4): Block Jacobi (per-block IC(0), with
 * PCG or with BiCGSTAB, the Krylov method Sec. 4.3 pairs with it) and
 * bordered block diagonal (per-block ILU(0) + dense Schur complement of the
 * border, GMRES(m)).  Both build the preconditioner from the numerics-
 * based filter (Eq. filter) and the diagonal correction (Eq. diagcorr).
 *
 * Conventions shared by every entry point:
 *   - Sparse matrices are CSR: int64 row pointers (nrows+1 entries), int32
 *     column indices sorted strictly ascending inside each row (no
 *     duplicates), double values.  Violations return SDSL_ERR_ARG.
 *   - Pointers named in sdsl_options.mem_space are either all host or all
 *     device pointers; block pointers are always host arrays.
 *   - Every call returns a status code; nothing is thrown across the ABI.
 *     sdsl_last_error() gives a message for the calling thread.
 *   - Calls on one handle are ordered on the handle's stream and are not
 *     thread-safe; different handles may be used from different threads.
 *   - The handle owns all device memory it allocates, until sdsl_free.  The
 *     caller keeps ownership of every array it passes; setup copies them.
 */
#ifndef SDSL_H
#define SDSL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdsl_handle_s* sdsl_handle;
typedef struct sdsl_batch_s* sdsl_batch;

typedef enum {
  SDSL_OK = 0,
  SDSL_ERR_ARG = 1,           /* bad size, pointer, option or CSR structure */
  SDSL_ERR_OOM = 2,           /* device allocation failed */
  SDSL_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  SDSL_ERR_BREAKDOWN = 4,     /* factor pivot not positive/finite after every shift, or Krylov breakdown */
  SDSL_ERR_NOT_CONVERGED = 5, /* maxit reached; x holds the last iterate */
  SDSL_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
  SDSL_ERR_STATE = 7          /* call out of order (e.g. solve before factor) */
} sdsl_status;

enum { SDSL_FORM_CSR = 0, SDSL_FORM_NORMAL = 1, SDSL_FORM_AUGMENTED = 2 };
/* SDSL_BJ_BICGSTAB: right-preconditioned BiCGSTAB (van der Vorst 1992; right
 * preconditioning as in Sec. 2.2) with the Block-Jacobi preconditioner of
 * SDSL_BJ_PCG, on the same forms (normal or CSR).  stats.iters counts passes
 * (two products and two preconditioner applies each); a pass whose first
 * half meets the tolerance ends there.  Breakdown (a zero or non-finite
 * rt.v, t.t, omega or rho) returns SDSL_ERR_BREAKDOWN. */
/* SDSL_BBD_GCR: restarted right-preconditioned GCR(m) (the paper's IGCR(m)
 * paired with BBD in Sec. 4.2-4.3, read as the GCR of Eisenstat, Elman and
 * Schultz 1983) with the BBD preconditioner of SDSL_BBD_GMRES, on the
 * augmented form; m = restart.  Each step: p = M^{-1} r, q = K p, q and p
 * orthogonalised against the step's earlier q (modified Gram-Schmidt, the
 * same coefficients applied to p), normalised by ||q||; x += (q^T r) p,
 * r -= (q^T r) q.  A cycle starts from the true residual.  stats.iters
 * counts products; a zero or non-finite ||q|| returns SDSL_ERR_BREAKDOWN. */
enum { SDSL_BJ_PCG = 0, SDSL_BBD_GMRES = 1, SDSL_BJ_BICGSTAB = 2, SDSL_BBD_GCR = 3 };
enum { SDSL_MEM_HOST = 0, SDSL_MEM_DEVICE = 1 };

typedef struct {
  int form;                      /* SDSL_FORM_*: what sdsl_setup receives */
  int method;                    /* SDSL_BJ_PCG, SDSL_BJ_BICGSTAB (Sec. 2.3), SDSL_BBD_GMRES or
                                    SDSL_BBD_GCR (Sec. 2.4) */
  int64_t nblocks;               /* number of diagonal blocks (Sec. 2.3 "partition") */
  const int64_t* block_ptr;      /* host, nblocks+1 row offsets of the blocks; NULL = equal split.
                                    Augmented form: row blocks of A (last entry = m - border) */
  const int64_t* col_block_ptr;  /* host, augmented form only: column blocks of A (nblocks+1) */
  int64_t border;                /* augmented form: number of linking rows of A (the last rows) */
  double tau;                    /* filter threshold of Eq. (filter), >= 0; 1e-3 in Sec. 3.2 */
  double delta;                  /* diagonal correction of Eq. (diagcorr), >= 0; 1e-12 in Sec. 3.3 */
  double rho;                    /* regularisation: rho*I added to S (normal) or the (2,2) block (augmented) */
  int factor_prec;               /* storage of the factors: 64, 32 or 16 (BF16; Block Jacobi with the staged
                                    solves only -- a trial of the coarsest storage); the Krylov loop is FP64 */
  double rtol;                   /* relative residual target ||b - A x|| / ||b|| (1e-8 in Sec. 4) */
  int64_t maxit;                 /* iteration cap (products with the system matrix) */
  int restart;                   /* GMRES restart length m */
  double refactor_ratio;         /* reuse rule (Sec. 3.4): rebuild before the next solve when a converged
                                    solve needs more than ratio * the iterations of the first converged solve
                                    after the last build, or when a solve does not converge; a solve that does
                                    not converge under a reused preconditioner is repeated after a rebuild in
                                    the same call.  0 disables automatic rebuilds */
  int mem_space;                 /* SDSL_MEM_HOST or SDSL_MEM_DEVICE for matrix/vector pointers */
  void* stream;                  /* cudaStream_t to order all work on; NULL = the legacy default stream */
  int graph_iters;               /* Krylov iterations captured per CUDA graph launch; 0 = no graphs
                                    (BiCGSTAB captures at most 4 passes: the applies and products of
                                    passes after the converged one still run) */
  int tune;                      /* 1 (default) = autotune: time candidate launch shapes on the handle's own
                                    matrix -- the PCG product's form and lanes per row, the staged sweeps'
                                    tile shape -- and keep the fastest (a candidate must beat the default by
                                    5 %).  The choice is cached per structure (sizes of A and S, blocks,
                                    method, precisions) for the life of the process: the first
                                    factorization of a structure pays the timing, later ones reuse it.
                                    Options set explicitly (spmv_form, sweep_lane_entries, sweep_far_gap)
                                    are kept.  0 = the built-in heuristics */
  int profile;                   /* 1 = time every Krylov kernel with CUDA events (no graphs; slower) */
  int apply_prec;                /* arithmetic of the triangular solves with FP32 factors: 32 (FP32),
                                    48 (float-float: pairs of FP32 numbers with error-free products and
                                    compensated sums, linear to ~1e-14; staged solves only) or 64 (FP64);
                                    0 = auto: 48 with FP32 factors where the staged solves run, else 64.
                                    FP64 factors are always applied in FP64 */
  int flexible;                  /* PCG beta: 0 = rho_new/rho, 1 = flexible z_new^T(r_new - r_old)/rho
                                    (robust to an FP32 apply); -1 = 1 iff the apply is FP32 */
  int solve_kernel;              /* block triangular solves: 0 auto, 1 level-synchronous (barrier per
                                    level), 2 flag-synchronised (rows in level order, readiness of every
                                    value in shared memory; needs the block to fit in shared memory),
                                    3 staged: level tiles copied into shared memory ahead of use
                                    (cp.async) by 16 warps per block (blocks of at most 65,535 rows) */
  int spmv_form;                 /* PCG product S p (normal form): 0 auto (fewer HBM bytes; sliced ELL copies
                                    of A and A^T when their padding is small), 1 explicit CSR of S,
                                    2 factored A (theta o (A^T p)) + rho p on CSR, 3 factored on sliced ELL */
  int orthog;                    /* GMRES orthogonalization: 0 modified Gram-Schmidt, 1 classical twice */
  int sweep_warps;               /* warps per block that run the staged triangular sweeps: 0 auto, 1..16 */
  int sweep_backoff_ns;          /* sleep between unsuccessful readiness polls in those sweeps: -1 auto, 0..1000 */
  int sweep_lane_entries;        /* tile shape of those sweeps: a row gets the fewest lanes (a power of two)
                                    that leave at most this many of its entries per lane; 0 auto, 1..64 */
  int schur_lu;                  /* BBD border Schur LU: 0 auto (blocked, trailing update on tensor cores),
                                    1 blocked on CUDA cores, 2 unblocked (one column per step) */
  int sweep_wait;                /* readiness in those sweeps: 0 auto (2), 1 per value (a tile waits until
                                    every value it reads is solved), 2 per level (a tile's far entries wait, parked on an mbarrier, until the
                                    level sweep_far_gap below is complete; its near entries per value),
                                    3 level-synchronous (the block's warps step through its levels together,
                                    one named barrier per level; no waits inside a level) */
  int wait_limit;                /* polls after which a wait in those sweeps gives up and the solve returns
                                    SDSL_ERR_TIMEOUT; 0 = default (2^23 polls, about a second; 1,024 under
                                    wait_test) */
  int sweep_far_gap;             /* tile shape of the staged sweeps: entries whose column lies at least this
                                    many levels below the row are summed first, behind one wait on a level
                                    count; the nearer ones are read by the row's first lane last, polling
                                    the values; 0 = auto (3, or tuned), else 2..16; 1 (every entry far)
                                    only with sweep_wait 1.  The level-synchronous sweep uses 1 */
  int64_t tau_switch_step;       /* two-phase filter (Sec. 4.3): from this IPM step on (counted in
                                    sdsl_update_diag calls) builds filter with tau_after; 0 = off */
  double tau_after;              /* the second phase's threshold (1e-2 in Sec. 4.3) */
  double tau_relax;              /* filter relaxation (Sec. 4.3): a solve that does not converge under a
                                    freshly built preconditioner is repeated once after a rebuild with
                                    threshold tau * tau_relax; later builds use the scheduled tau again.
                                    0 = off, else in (0, 1) */
  int sweep_slots;               /* ring depth (tiles per warp in flight) of the staged sweeps: 0 = the deepest
                                    that fits shared memory, else 2..4.  Handles solved together by
                                    sdsl_batch_solve must share it (with the precisions and lane entries) */
  int wait_test;                 /* 1 = exercise the timeout path: every per-level wait of the staged sweeps
                                    waits for one tile more than its level has, which never arrives, so
                                    each wait gives up after wait_limit polls (no fault, the context stays
                                    usable) and the solve returns SDSL_ERR_TIMEOUT.  0 in normal use */
} sdsl_options;

typedef struct {
  int64_t iters;          /* Krylov iterations of the last solve: products with the system matrix
                             (PCG, GMRES) or BiCGSTAB passes */
  int64_t restarts;       /* PCG true-residual restarts / GMRES cycles */
  int rebuilt;            /* 1 if the last solve was preceded by an automatic rebuild */
  int status;             /* sdsl_status of the last solve */
  double rel_res_true;    /* ||b - A x|| / ||b|| recomputed in FP64 at exit */
  double rel_res_rec;     /* recurrence (or GMRES estimate) residual at exit */
  double ms_setup, ms_factor, ms_solve, ms_update;   /* device time of the last call of each kind */
  int64_t n;              /* system dimension */
  int64_t nnz_system;     /* nnz of S or K */
  int64_t nnz_precond;    /* nnz of the filtered, corrected preconditioner matrix P */
  int64_t nnz_factor;     /* nnz of the triangular factor(s) used per application */
  int64_t levels_lower, levels_upper;   /* total level count over blocks */
  int64_t max_levels;     /* largest per-block level count */
  int64_t shifted_blocks; /* blocks that needed a diagonal shift to factor */
  int64_t builds;         /* factorizations since setup */
  double bytes_per_iter;  /* algorithmic HBM bytes of one Krylov iteration (model) */
  double kernel_ms[4];    /* profile mode: summed device time of the iteration kernels:
                             [0] SpMV + p^T q, [1] update + preconditioner, [2] direction, [3] other */
  int64_t kernel_launches[4];
  double kernel_bytes[4]; /* algorithmic HBM bytes per launch of the kernels above (model) */
  int64_t spmv_lanes;     /* lanes per row of the SpMV in use */
  int64_t solve_lanes;    /* lanes per row of the block triangular solves in use */
  int64_t tuned_spmv_lanes; /* explicit-S SpMV lanes chosen by the autotuner (0 if it did not run) */
  int64_t product_lanes[2]; /* factored normal-equation product: lanes per row of A^T p and of A u
                               on CSR, -1 on the sliced ELL copies (0 when the explicit S is used) */
  double ms_schur;        /* BBD: device time of the border Schur complement assembly (part of ms_factor) */
  double ms_dense_lu;     /* BBD: device time of its dense FP32 LU (part of ms_factor) */
  double ms_dense_inverse; /* BBD: device time of the explicit FP32 inverse from that LU (part of ms_factor) */
  double tau_used;         /* filter threshold of the preconditioner the last solve used */
  double ms_tune;          /* host time the autotuner spent in the last factorization (0 when its choice
                              for this structure was already cached) */
  int64_t sweep_shape[2];  /* staged sweeps' tile shape in use: entries per lane, far gap */
  int64_t product_kind;    /* PCG product chosen by the autotuner: 1 explicit S, 2 factored CSR, 3 factored
                              sliced ELL (0: not tuned) */
  int64_t iters_discarded; /* iterations of a first attempt of the last solve that did not converge under a
                              reused preconditioner and was repeated after a rebuild (0 if none); ms_solve
                              covers both attempts */
} sdsl_stats;

typedef struct {
  int64_t n, nnz_system, nnz_precond, nblocks, border;
  int64_t levels_lower, levels_upper;
  int factored;
  int64_t device_bytes;       /* device memory the handle holds now (its arenas) */
  int64_t peak_device_bytes;  /* the most it has held at once, temporaries of setup and factor included */
} sdsl_info;

/* Fill *o with the defaults: BJ-PCG, normal form, tau 1e-3, delta 1e-12,
 * rho 1e-6, FP64 factors, rtol 1e-8, maxit 2000, restart 30, refactor_ratio
 * 1.5, device pointers, default stream, graph_iters 16, tune 1, profile 0,
 * apply_prec 0 (= factor_prec), flexible -1 (auto), solve_kernel 0 (auto), spmv_form 0 (auto),
 * orthog 0 (modified Gram-Schmidt). */
void sdsl_default_options(sdsl_options* o);

/* Create a handle and form the system matrix on the device.
 *   SDSL_FORM_NORMAL:    A is m x n (rowptr/col/val), theta has n entries;
 *                        S = A diag(theta) A^T + rho I (Eq. schur), dimension m.
 *                        The pattern of S (symbolic product) is computed once
 *                        here; the values again on every sdsl_update_diag.
 *                        Rounding of S_ij, h = max(i,j), l = min(i,j): sum over
 *                        shared columns k ascending of fma(fl(a_hk theta_k), a_lk, acc)
 *                        from +0, then S_ii + rho; S is exactly symmetric.
 *   SDSL_FORM_AUGMENTED: A is m x n with rows grouped by block and the
 *                        options.border linking rows last, columns grouped by
 *                        block; K (Eq. augmented) of dimension n+m is assembled
 *                        in bordered block-diagonal order (Sec. 2.4): for each
 *                        block its x unknowns then its lambda unknowns, border last.
 *   SDSL_FORM_CSR:       the n x n system matrix is given directly (m = n);
 *                        theta must be NULL.  For BJ-PCG it must be symmetric.
 * Errors: SDSL_ERR_ARG (NULL/negative sizes, bad block pointers, unsorted
 * CSR), SDSL_ERR_OOM, SDSL_ERR_CUDA.  *out is NULL on error. */
sdsl_status sdsl_setup(const sdsl_options* opt, int64_t m, int64_t n, const int64_t* rowptr,
                       const int32_t* col, const double* val, const double* theta, sdsl_handle* out);

/* Build the preconditioner from the current system values (Algorithms 2-3):
 * filter (Eq. filter, scope: inside the diagonal blocks for Block Jacobi, the
 * whole matrix for BBD), diagonal correction (Eq. diagcorr), level sets of the
 * block triangular solves, per-block IC(0) (BJ) or ILU(0) (BBD) with the
 * shift-retry rule (a block whose factor breaks down is refactored with
 * diagonal p_ii + alpha p_ii, alpha = 1e-3, 1e-2, 1e-1, 1), and for BBD the
 * dense Schur complement of the border and its LU.  Errors: SDSL_ERR_BREAKDOWN
 * if a block fails with every shift. */
sdsl_status sdsl_factor(sdsl_handle h);

/* Solve A x = b to options.rtol (Krylov loop in FP64 on the device).  b and x
 * have the system dimension and live in options.mem_space; x is the initial
 * guess on entry unless x0_zero != 0, and the solution on exit.  With a reuse
 * rule set (refactor_ratio > 0, Sec. 3.4): if the last solve requested a
 * rebuild the preconditioner is rebuilt first; if this solve does not
 * converge under a preconditioner that earlier solves already used, the
 * preconditioner is rebuilt from the current system and the solve repeated
 * from the same initial guess (st->rebuilt = 1, st->iters_discarded = the
 * first attempt's iterations).  st may be NULL.  Errors: SDSL_ERR_STATE before
 * sdsl_factor, SDSL_ERR_NOT_CONVERGED (x = last iterate), SDSL_ERR_BREAKDOWN. */
sdsl_status sdsl_solve(sdsl_handle h, const double* b, double* x, int x0_zero, sdsl_stats* st);

/* Continuous batching of independent solves (the serving loop): a batch
 * holds requests -- factored handles with their b and x -- whose Block-Jacobi
 * PCG iterations advance together in the same persistent launches (the
 * factored product, the update with the staged block sweeps, the direction)
 * over a device table of (request, block) items, graph_iters iterations per
 * CUDA graph (Sec. 2.3: the blocks are independent, so blocks of different
 * systems are too).  Every request keeps its own grids, partial sums and
 * scalars, so its iterates, count and result are those of sdsl_solve on it
 * alone, bit for bit; the reuse rule and the filter relaxation act per
 * request as in sdsl_solve.  Requests join with sdsl_batch_add and leave when
 * their solve ends: sdsl_batch_step launches the batch until at least one
 * request has finished (or max_graphs graph launches), then hands back up to
 * cap finished handles (done_h) with their statistics (done_st, may be NULL)
 * -- x holds the result on the handle's stream -- and they leave the batch;
 * requests still running stay.  The launch tables and graph are rebuilt when
 * the membership changes.  A handle fits a batch when it uses Block-Jacobi
 * PCG with the staged sweeps and the factored product on the sliced ELL
 * copies, on the batch's device, with the factor and apply precision, ring
 * depth (sweep_slots) and lane entries of the batch's other members
 * (SDSL_ERR_ARG otherwise).  While a handle is in a batch, make no other
 * call on it.  One thread drives a batch; sdsl_batch_free abandons members
 * still running (their x is not written). */
sdsl_status sdsl_batch_create(int graph_iters, sdsl_batch* out);
sdsl_status sdsl_batch_add(sdsl_batch batch, sdsl_handle h, const double* b, double* x, int x0_zero);
sdsl_status sdsl_batch_step(sdsl_batch batch, int max_graphs, sdsl_handle* done_h, sdsl_stats* done_st, int cap,
                            int* ndone);
int sdsl_batch_size(sdsl_batch batch);
sdsl_status sdsl_batch_free(sdsl_batch batch);

/* Solve count independent systems together, each on its own factored handle
 * (a batch of sdsl_batch_create / _add / _step until all have finished, with
 * the first handle's graph_iters).  hs[i], b[i], x[i] as in sdsl_solve
 * (x0_zero shared); st may be NULL, else count entries.  The handles must be
 * distinct and factored; they are solved together when every one fits one
 * batch (see above), otherwise one after another.  Returns SDSL_OK if every
 * solve succeeded, else the first failing status (each in st[i].status). */
sdsl_status sdsl_batch_solve(int count, sdsl_handle* hs, const double* const* b, double* const* x, int x0_zero,
                             sdsl_stats* st);

/* New IPM scaling theta (Sec. 3.4 preconditioner reuse): recompute the system
 * values on the device (normal: S on its fixed pattern; augmented: the x
 * diagonal -1/theta), keep the factors.  theta has n entries in mem_space.
 * SDSL_ERR_STATE for SDSL_FORM_CSR. */
sdsl_status sdsl_update_diag(sdsl_handle h, const double* theta);

/* Filter threshold tau (Eq. filter) of the next preconditioner build (the
 * factorization of sdsl_factor or of an automatic rebuild): the hook for an
 * IPM driver's own tau schedule (Sec. 4.2 relaxes and re-tightens it across
 * IPM steps; Sec. 4.3 switches it once).  The current preconditioner is kept
 * until the next build.  Errors: SDSL_ERR_ARG for tau < 0 or NaN. */
sdsl_status sdsl_set_tau(sdsl_handle h, double tau);

/* Release everything the handle owns (stream-ordered).  NULL-safe. */
sdsl_status sdsl_free(sdsl_handle h);

/* Statistics of the handle (counters of the last calls). */
sdsl_status sdsl_get_stats(sdsl_handle h, sdsl_stats* st);
sdsl_status sdsl_get_info(sdsl_handle h, sdsl_info* info);

/* Copy-outs for verification (host buffers, sizes from sdsl_get_info):
 *  sdsl_export_system: the system matrix (n+1, nnz_system, nnz_system);
 *  sdsl_export_precond: P after filter+correction (n+1, nnz_precond x2) and
 *    the factor values on P's layout (IC(0): l_ij at j <= i; ILU(0): unit-L
 *    multipliers at j < i, U at j >= i; factor_prec 32 exports the stored
 *    FP32 values widened), plus the shift alpha used per block (nblocks);
 *    any output pointer may be NULL;
 *  sdsl_export_levels: which = 0 lower / 1 upper; nlev[nblocks] levels per
 *    block, level_ptr[levels+1] offsets into level_rows[n] (rows ascending
 *    inside a level, blocks in order);
 *  sdsl_export_schur: BBD only, the dense border Schur complement (FP64,
 *    row-major border x border). */
sdsl_status sdsl_export_system(sdsl_handle h, int64_t* rowptr, int32_t* col, double* val);
sdsl_status sdsl_export_precond(sdsl_handle h, int64_t* rowptr, int32_t* col, double* pval, double* fval,
                                double* alpha);
sdsl_status sdsl_export_levels(sdsl_handle h, int which, int32_t* nlev, int64_t* level_ptr, int32_t* level_rows);
sdsl_status sdsl_export_schur(sdsl_handle h, double* sb);

/* BBD only (Sec. 2.4, the dense border factorization): the LU's pivot rows
 * (ipiv[k] = row swapped with row k at step k, border-local, border entries)
 * and its pivots u_kk in FP64 (the blocked LU, schur_lu 0 or 1, chooses and
 * keeps them in FP64; the unblocked one, schur_lu 2, gives its FP32 u_kk
 * widened).  Host buffers; either may be NULL. */
sdsl_status sdsl_export_schur_lu(sdsl_handle h, int32_t* ipiv, double* pivots);

/* y = A x with the handle's system matrix (device pointers, FP64). */
sdsl_status sdsl_spmv(sdsl_handle h, const double* x, double* y);

/* z = M^{-1} r with the current preconditioner (device pointers, FP64). */
sdsl_status sdsl_precond_apply(sdsl_handle h, const double* r, double* z);

/* Largest n accepted by sdsl_normal_spmv_noalloc: its static scratch holds
 * this many doubles (4 MiB) on every GPU where the library is loaded. */
#define SDSL_NOALLOC_MAX_COLS (1 << 19)

/* y = A (theta o (A^T x)) + rho x, the normal-equation product of
 * sdsl_spmv without forming S and without allocating.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- a host program whose memory manager has reserved nearly all
 * of HBM for its own pool, or a latency-bound serving loop where an
 * allocation would synchronise the device -- and therefore cannot create a
 * handle.
 *   m, n       A is m x n; 0 <= n <= SDSL_NOALLOC_MAX_COLS, else SDSL_ERR_ARG
 *              with nothing launched.
 *   nnz        nonzeros of A (chooses lanes per row; must fit int32).
 *   a_*        A in CSR: rowptr[m+1] (int64), col/val[nnz]; at_* A^T in CSR
 *              (rowptr[n+1]).  Valid CSR with columns in range is the
 *              caller's responsibility: it is not checked here.
 *   theta[n], x[m], y[m]: device memory of the current device (or managed),
 *              owned by the caller; y is overwritten, x and y may not alias.
 *   stream     cudaStream_t (NULL: the legacy default stream); the call only
 *              enqueues work and returns without synchronising.
 * The intermediate theta o (A^T x) lives in a file-scope __device__ array
 * of SDSL_NOALLOC_MAX_COLS doubles.  The first call on a device (and the
 * first after its context was re-created, e.g. by cudaDeviceReset) looks up
 * that array's address with the device current (the library's module is
 * loaded then if it was not yet), so make that call before any stream
 * capture begins.  All calls share the array: calls whose kernels
 * overlap on the GPU (different streams without ordering between them) race
 * on it.  Each call writes every scratch entry it reads, so nothing carries
 * over between calls.  Errors: SDSL_ERR_ARG for bad sizes, NULL pointers or
 * pointers that are not device memory of the current device; SDSL_ERR_CUDA
 * for a failed lookup or launch (sdsl_last_error() has the text). */
sdsl_status sdsl_normal_spmv_noalloc(int64_t m, int64_t n, int64_t nnz, const int64_t* a_rowptr,
                                     const int32_t* a_col, const double* a_val, const int64_t* at_rowptr,
                                     const int32_t* at_col, const double* at_val, const double* theta, double rho,
                                     const double* x, double* y, void* stream);

/* Number of kernels this library has launched in the process so far (every
 * launch, including those inside CUDA graphs, counted once). */
int64_t sdsl_kernel_launches(void);

const char* sdsl_status_str(sdsl_status s);
const char* sdsl_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SDSL_H */
