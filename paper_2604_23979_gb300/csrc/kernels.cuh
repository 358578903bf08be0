// kernels.cuh -- host launchers of the device kernels (internal interface
// between the C ABI in api.cu and the kernel translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sdsl {

// ---- setup.cu: system formation (Eq. schur / Eq. augmented)
cudaError_t check_csr(int64_t nrows, int64_t ncols, const int64_t* rp, const int32_t* ci, int* bad, cudaStream_t st);
cudaError_t transpose_csr(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v, int64_t* trp,
                          int32_t* tci, double* tv, int64_t* scan_scratch, cudaStream_t st);
cudaError_t transpose_fill(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                           const int64_t* trp, int32_t* tci, double* tv, int64_t* cursor, cudaStream_t st);
cudaError_t sort_rows(int64_t nrows, const int64_t* rp, int32_t* ci, double* v, cudaStream_t st);
cudaError_t normal_symbolic_count(int64_t m, const int64_t* rp, const int32_t* ci, const int64_t* trp,
                                  const int32_t* tci, int64_t* srp, int32_t* long_rows, int32_t* nlong,
                                  cudaStream_t st);
cudaError_t normal_symbolic_long(bool fill, int nlong, const int32_t* long_rows, const int64_t* rp,
                                 const int32_t* ci, const int64_t* trp, const int32_t* tci, int64_t* srp,
                                 int32_t* sci, int* err, cudaStream_t st);
cudaError_t normal_symbolic_fill(int64_t m, const int64_t* rp, const int32_t* ci, const int64_t* trp,
                                 const int32_t* tci, const int64_t* srp, int32_t* sci, cudaStream_t st);
cudaError_t normal_values(int64_t m, const int64_t* rp, const int32_t* ci, const double* v, const int64_t* trp,
                          const int32_t* tci, const double* tv, const double* theta, double rho,
                          const int64_t* srp, const int32_t* sci, double* sv, cudaStream_t st);
cudaError_t bbd_positions(int64_t m, int64_t n, int64_t nblocks, const int64_t* rbp, const int64_t* cbp,
                          const int64_t* kbp, int64_t* pos, cudaStream_t st);
cudaError_t augmented_count(int64_t m, int64_t n, const int64_t* rp, const int64_t* trp, const int64_t* pos,
                            int64_t* krp, cudaStream_t st);
cudaError_t augmented_fill(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                           const int64_t* trp, const int32_t* tci, const double* tv, const double* theta, double rho,
                           const int64_t* pos, const int64_t* krp, int32_t* kci, double* kv, int64_t* xdiag,
                           cudaStream_t st);
cudaError_t augmented_theta(int64_t n, const double* theta, const int64_t* xdiag, double* kv, cudaStream_t st);

// ---- precond.cu: filter (Eq. filter), correction (Eq. diagcorr), levels, factors
cudaError_t diag_values(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, double* d, cudaStream_t st);
// whole = 0: keep in-block entries only (Block Jacobi); 1: every entry (BBD)
cudaError_t filter_count(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* d,
                         const int32_t* row_block, const int64_t* bp, int whole, double tau, int64_t* prp,
                         cudaStream_t st);
cudaError_t filter_fill(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* d,
                        const int32_t* row_block, const int64_t* bp, int whole, double tau, double delta,
                        const int64_t* prp, int32_t* pci, double* pv, int64_t* pdiag, cudaStream_t st);
cudaError_t row_blocks(int64_t n, int64_t nblocks, const int64_t* bp, int32_t* row_block, cudaStream_t st);
cudaError_t mirror_map(int64_t n, const int64_t* prp, const int32_t* pci, const int64_t* pdiag, int64_t* mir,
                       int* bad, cudaStream_t st);
// Level sets of the in-block lower (dir = 0) or upper (dir = 1) triangle.
cudaError_t levels(int dir, int64_t nblocks, const int64_t* bp, const int64_t* prp, const int32_t* pci,
                   const int64_t* pdiag, int32_t* cnt, int32_t* lev, int32_t* fa, int32_t* fb, int32_t* nlev,
                   cudaStream_t st);
cudaError_t level_lists(int64_t nblocks, const int64_t* bp, const int32_t* lev, const int32_t* lev_off,
                        int32_t* hist, int32_t* level_ptr, int32_t* level_rows, cudaStream_t st);
// IC(0) of every block with every shift of the retry ladder at once: CTA
// (b, t) writes block b's factor for alpha[t] into Fall + t*nnz, dinv_all +
// t*n, and status[b*nshift + t] (1 = breakdown).  pick_shift copies the
// chosen shift's factor of each block into F / dinv.
cudaError_t ic0_factor_all(int64_t nblocks, const int64_t* bp, const int64_t* prp, const int32_t* pci,
                           const double* pv, const int64_t* pdiag, const int32_t* lev_off, const int32_t* level_ptr,
                           const int32_t* level_rows, const double* alpha, int nshift, int64_t nnz, int64_t n,
                           double* Fall, double* dinv_all, int32_t* status, const int32_t* order,
                           cudaStream_t st);
cudaError_t pick_shift(const int64_t* bp, const int64_t* prp, const int32_t* choice, int64_t nnz, int64_t n,
                       const double* Fall, const double* dinv_all, double* F, double* dinv, const int32_t* rb,
                       int64_t nrows, cudaStream_t st);
cudaError_t ilu0_factor(int64_t nblocks, const int64_t* bp, const int64_t* prp, const int32_t* pci, const double* pv,
                        const int64_t* pdiag, const int32_t* lev_off, const int32_t* level_ptr,
                        const int32_t* level_rows, const double* alpha, const int32_t* active, double* F,
                        double* dinv, int32_t* status, cudaStream_t st);
// IC(0): copy l_ji to the upper position (i, j); make the FP32 copies.
cudaError_t ic0_finish(int64_t n, int64_t nnz, const int64_t* prp, const int64_t* pdiag, const int64_t* mir,
                       double* F, const double* dinv, float* Ff, float* dinvf, cudaStream_t st);
cudaError_t to_float(int64_t n, const double* a, float* b, cudaStream_t st);
cudaError_t round_bf16(int64_t n, float* a, cudaStream_t st);
// Variable-width tiles (see precond.cu): fill the stream from a host-built plan.
// lev: level of every row within its block for this direction (far entries
// of a row at level L have column level <= L - gap, near ones above that).
// tile_meta: 3 ints per tile (level, tiles of level L - 1, tiles of level
// L - gap).  *bad = 1 if a row has more than 255 near entries.
cudaError_t vt_fill(int dir, int64_t ntiles, const int32_t* tile_rows_ptr, const int32_t* plan_rows,
                    const int8_t* plan_logv, const int32_t* row_block, const int64_t* bp, const int64_t* prp,
                    const int32_t* pci, const int64_t* pdiag, const double* F, const double* dinv, const int32_t* lev,
                    int prec, const int64_t* toff, const int32_t* tile_meta, unsigned char* stream, int* bad,
                    int gap, cudaStream_t st);
// Dynamic shared memory of the staged solve kernel (sweep.cu): y in both
// directions, the warps' tile rings, the block's staged tile offsets and
// its per-level completion counters.
size_t staged_smem_bytes(int64_t max_block, size_t tc_size, int warps, int slot_bytes, int slots, int64_t max_tiles,
                         int64_t max_levels);


// ---- krylov.cu: SpMV, PCG iteration kernels, residuals
struct PcgState {
  double rho;      // r^T z of the current direction
  double alpha;    // step of the current iteration
  double beta;
  double pq;       // p^T q
  double rr;       // ||r||^2 after the update
  double rz_new;
  double tol2;     // (rtol * ||b||)^2
  double tr;       // ||b - A x||^2 of the last true-residual check
  long long iters;
  long long maxit;
  int done;        // 0 running, 1 recurrence converged, 2 maxit, 3 breakdown
  int err;         // 1 = a bounded device wait gave up (SDSL_ERR_TIMEOUT)
  double zq;       // z_new^T q (flexible beta)
  unsigned int ticket[4];
};

// Device scalars of BiCGSTAB (bicgstab.cu); iters, alpha, done, err, tol2
// and rr live in the solve's PcgState.
constexpr int kBicgMaxCtas = 152 * 4;
struct BicgScalars {
  double rho;      // rt . r of the current pass
  double omega, beta;
  double rv, ts, tt;
  double* part;    // 2 x kBicgMaxCtas partial sums
  long long maxit;
  int first;       // 1: the next pass starts with p = r
  unsigned int ticket;
};

struct TriSolve {  // block triangular factors on the layout of P
  int64_t nblocks;
  const int64_t* bp;
  const int64_t* prp;
  const int32_t* pci;
  const int64_t* pdiag;
  const double* F;      // FP64 factor values (lower: L, upper: L^T or U)
  const float* Ff;      // FP32 copy (factor_prec 32)
  const double* dinv;   // 1/l_ii (IC) or 1/u_ii (ILU)
  const float* dinvf;
  const int32_t* lev_off_lo;
  const int32_t* lev_ptr_lo;
  const int32_t* lev_rows_lo;
  const int32_t* lev_off_up;
  const int32_t* lev_ptr_up;
  const int32_t* lev_rows_up;
  int unit_lower;       // 1 for ILU(0) (L has a unit diagonal)
  int prec;             // storage of the factor values: 64, 32 or 16 (BF16, staged solves only)
  int lanes;            // lanes per row in the solves (2..32)
  int64_t max_block;    // largest block (rows) -> shared-memory staging if it fits
  float* yscratch;      // global staging when the block does not fit in shared memory
  double* yscratch64;
  // Level-ordered packed copies of the strict triangles for the flag-
  // synchronised solves: position q of block b (row lev_rows[q]) owns entries
  // [off[q], off[q+1]) with block-local columns; values and inverse diagonal in
  // the storage precision (float or double).
  const int64_t* fwd_off;
  const int32_t* fwd_col;
  const void* fwd_val;
  const void* fwd_dinv;
  const int32_t* fwd_row;   // block-local row of position q
  const int64_t* bwd_off;
  const int32_t* bwd_col;
  const void* bwd_val;
  const void* bwd_dinv;
  const int32_t* bwd_row;
  const int64_t* fwd_pos;   // per block: first position of its padded schedule (nblocks+1)
  const int64_t* bwd_pos;
  // staged tile streams (solve_kernel 3): tile t of a direction is the
  // byte range [toff[t], toff[t+1]) of the stream; block b owns tiles
  // tile_ptr[b] .. tile_ptr[b+1]-1.
  const unsigned char* fwd_stream;
  const int64_t* fwd_toff;
  const int64_t* fwd_tile;
  const unsigned char* bwd_stream;
  const int64_t* bwd_toff;
  const int64_t* bwd_tile;
  int staged;           // 1: staged level tiles (cp.async copies into a per-warp shared-memory ring)
  int slot_bytes;       // ring slot size; larger tiles are read from global memory directly
  int kreg;             // entries per lane and gather round of the staged solves (8 or 16)
  int level_wait;       // staged solves: 0 = per-value readiness, 1 = per-level mbarriers (far part) and
                        // per-value readiness (near part), 2 = level-synchronous (one named barrier per level)
  int max_levels;       // largest level count of a block (either direction): counters in shared memory
  int64_t max_tiles;    // max over blocks of (forward tiles + backward tiles): staged tile offsets
  int slots;            // ring slots per warp
  int sync_free;        // 1: packed flag-synchronised solves (block fits in shared memory)
  int apply_prec;       // arithmetic of the apply: 64 or 32
  int flexible;         // 1: beta = -alpha z_new^T q / rho (robust to an inexact FP32 apply)
  int threads;          // CTA size of the solve kernel
  int sweep_warps;      // warps of the staged solve that take tiles (the rest only stage and reduce)
  int backoff_ns;       // sleep between unsuccessful readiness polls
  int wait_limit;       // polls after which a staged-sweep wait gives up (sets the timeout flag)
  int wait_pad;         // 1: per-level waits wait for one tile more than exists (timeout-path test)
  int far_gap;          // staged tiles: entries at least this many levels below the row are "far"
  const int32_t* fwd_ltiles;  // staged tiles per level (forward), indexed like lev_off_lo: block b, level l
  const int32_t* bwd_ltiles;  // at lev_off_[lo|up][b] + l (backward)
  const int32_t* fwd_lend;    // tiles of block b through level l (cumulative), same indexing
  const int32_t* bwd_lend;
};

// Packed level-ordered triangle of one direction (dir 0 = strict lower in
// lower-level order, 1 = strict upper in upper-level order).  pack_count
// writes the entry count of every position into off[0..npos); the caller
// scans it into offsets; pack_fill copies columns (block-local), values and
// inverse diagonals (float if prec == 32 else double) and block-local rows.
// lev_rows here is the padded schedule: the global row of every position, or
// -1 for a padding position (levels are padded to whole warp tiles).
cudaError_t pack_count(int dir, int64_t npos, const int32_t* row_block, const int64_t* bp, const int64_t* prp,
                       const int32_t* pci, const int64_t* pdiag, const int32_t* lev_rows, int64_t* off,
                       cudaStream_t st);
cudaError_t pack_fill(int dir, int64_t npos, const int32_t* row_block, const int64_t* bp, const int64_t* prp,
                      const int32_t* pci, const int64_t* pdiag, const int32_t* lev_rows, const double* F,
                      const double* dinv, int prec, const int64_t* off, int32_t* col, void* val, void* pdinv,
                      int32_t* prow, cudaStream_t st);

// Sliced ELL copy of a CSR matrix (sell.cu): ranked rows perm, per slice of
// 32 ranked rows its width and its offset into col/val (slot-major).
struct SellMat {
  int64_t nrows, nslices;
  const int32_t* perm;
  const int64_t* off;
  const int32_t* wid;
  const int32_t* col;
  const double* val;
};

struct SpmvPlan {
  int64_t n;
  const int64_t* rp;
  const int32_t* ci;
  const double* v;
  int lanes;      // lanes per row (2..32)
  int grid;       // CTAs (fixed => deterministic partial sums)
  // factored form of the normal-equation operator, S p = A (theta o (A^T p)) + rho p
  int factored;   // 1: the PCG products use the factored form
  int64_t ncols;  // columns of A
  const int64_t* a_rp;  const int32_t* a_ci;  const double* a_v;    // A (m x n)
  const int64_t* at_rp; const int32_t* at_ci; const double* at_v;   // A^T (n x m)
  const double* theta;
  double rho;
  double* u;      // scratch, n entries
  int at_lanes, a_lanes;
  int at_grid;
  // rows longer than long_thr entries (e.g. the border rows of a BBD system,
  // which span every block) are summed by one CTA each before the row kernel
  // runs; the row kernel takes their values from long_ax.
  int long_thr;             // 0: no long rows
  int64_t n_long;
  const int32_t* long_rows; // ascending
  double* long_ax;          // n_long values of the last product
  // factored product on sliced ELL copies of A and A^T
  int sell;
  SellMat a_sell, at_sell;
  unsigned sell_a_grid, sell_at_grid;
};

// SELL-32 construction (sell.cu): rank rows within windows and compute the
// slice widths (cnt = width x 32, to be scanned into offsets), then fill.
cudaError_t sell_rank_widths(int64_t nrows, const int64_t* rp, int32_t* perm, int32_t* wid, int64_t* cnt,
                             cudaStream_t st);
cudaError_t sell_fill(int64_t nrows, const int64_t* rp, const int32_t* ci, const double* v, const int32_t* perm,
                      const int64_t* off, const int32_t* wid, int32_t* col, double* val, cudaStream_t st);
// Factored normal-equation product on the SELL copies (pcg: partial p^T q, alpha).
cudaError_t sell_factored_product(const SpmvPlan& A, const double* p, double* q, double* part, PcgState* s, int pcg,
                                  cudaStream_t st);
int sell_occupancy(int which);
unsigned sell_grid_for(int64_t nslices, int max_ctas);

cudaError_t spmv(const SpmvPlan& A, const double* x, double* y, cudaStream_t st);
cudaError_t time_spmv(const SpmvPlan& A, const double* x, double* y, int reps, float* ms, cudaStream_t st);
// q = A p, partial p^T q; last CTA: alpha = rho/pq, iters++.
// q = A (theta o (A^T p)) + rho p through the scratch A.u (n entries); with
// pcg = 1 also the partial p^T q and, in the last CTA, alpha = rho/pq, iters++;
// with pcg = 2 the product alone, skipped once s->done is set.
cudaError_t factored_product(const SpmvPlan& A, const double* p, double* q, double* part, PcgState* s, int pcg,
                             cudaStream_t st);
int product_occupancy(int kind, int lanes);
cudaError_t time_factored(const SpmvPlan& A, const double* p, double* q, int reps, float* ms_at, float* ms_a,
                          cudaStream_t st);
cudaError_t pcg_spmv(const SpmvPlan& A, const double* p, double* q, double* part, PcgState* s, cudaStream_t st);
// x += alpha p, r -= alpha q, z = M^{-1} r per block; last CTA: convergence, beta.
// part: 3 sections of nblocks partial sums [||r||^2 | r^T z | z^T q].
cudaError_t pcg_update_precond(const TriSolve& M, const double* p, const double* q, double* x, double* r, double* z,
                               double* part, PcgState* s, cudaStream_t st);
// PCG update + staged Block-Jacobi apply (solve_kernel 3); modes as pcg_update_precond.
cudaError_t update_staged(const TriSolve& M, const double* p, const double* q, double* x, double* r, double* z,
                          double* pp, double* part, PcgState* s, int mode, cudaStream_t st);
// Dynamic shared memory of the flag-synchronised solve for a block size.
size_t sf_smem_bytes(int64_t max_block, size_t tc_size);
// p = z + beta p
cudaError_t pcg_direction(int64_t n, const double* z, double* p, PcgState* s, cudaStream_t st);
// z = M^{-1} r (no update).  mode 1: also p_out = z, s->rho = r^T z, s->rr =
// ||r||^2 (PCG start / restart); mode 2: z only; mode 3: z only, skipped once s->done is set.
cudaError_t precond_apply(const TriSolve& M, const double* r, double* z, double* p_out, double* part, PcgState* s,
                          int mode, cudaStream_t st);
// t = b - A x, ||t||^2 -> s->tr; if write_r, r = t.
cudaError_t true_residual(const SpmvPlan& A, const double* b, const double* x, double* r, double* part,
                          PcgState* s, int write_r, cudaStream_t st);
// ||a||^2 -> *out; part holds up to 608 partials, *ticket must start at 0.
cudaError_t norm2_sq(int64_t n, const double* a, double* part, double* out, unsigned int* ticket, cudaStream_t st);
cudaError_t pcg_init_state(PcgState* s, double tol2, long long maxit, cudaStream_t st);

// ---- batched PCG iteration over several requests (sell.cu, sweep.cu,
// krylov.cu): the device descriptor of one request and a work item of a
// persistent launch (request, virtual CTA of that request's own grid).
struct BatchReq {
  TriSolve M;      // its preconditioner (staged sweeps)
  SpmvPlan A;      // its product (factored, sliced ELL)
  double *x, *r, *z, *p, *q;
  double* part;      // product partial sums (g_a entries)
  double* part_blk;  // update partial sums (3 x nblocks)
  PcgState* s;
  int64_t n;
  int g_at, g_a, g_dir;  // the request's grids of the product halves and the direction
};
struct BatchItem {
  int32_t req, vb;
};
cudaError_t batch_product(const BatchReq* reqs, const BatchItem* items_at, int n_at, const BatchItem* items_a,
                          int n_a, int grid, cudaStream_t st);
// M0: the first request's preconditioner (all must share the kernel shape:
// factor/apply precision, ring slots, entries per lane); smem: the largest
// request's dynamic shared memory.
cudaError_t batch_update(const TriSolve& M0, const BatchReq* reqs, const BatchItem* items, int nitems, int grid,
                         size_t smem, cudaStream_t st);
cudaError_t batch_direction(const BatchReq* reqs, const BatchItem* items, int nitems, int grid, cudaStream_t st);
size_t staged_smem_bytes_of(const TriSolve& M);
int direction_grid(int64_t n);

// ---- bicgstab.cu: the vector steps of right-preconditioned BiCGSTAB
cudaError_t bicg_init(BicgScalars* c, long long maxit, cudaStream_t st);
// rt = r, rho = r . r, first pass next (a start or a restart).
cudaError_t bicg_restart(int64_t n, const double* r, double* rt, BicgScalars* c, cudaStream_t st);
cudaError_t bicg_direction(int64_t n, const double* r, const double* v, double* p, const PcgState* s,
                           const BicgScalars* c, cudaStream_t st);
cudaError_t bicg_alpha(int64_t n, const double* rt, const double* v, PcgState* s, BicgScalars* c, cudaStream_t st);
cudaError_t bicg_omega(int64_t n, const double* t, const double* sv, PcgState* s, BicgScalars* c, cudaStream_t st);
cudaError_t bicg_finish(int64_t n, const double* sh, const double* t, const double* rt, double* x, double* r,
                        PcgState* s, BicgScalars* c, cudaStream_t st);

// ---- bbd.cu: BBD Schur complement, dense border LU, BBD apply, GMRES helpers
cudaError_t schur_init(int64_t nb, int64_t b0, const int64_t* prp, const int32_t* pci, const double* pv, double* SB,
                       cudaStream_t st);
int64_t schur_tiles(int64_t nb);
// One interior block of a Schur wave: rows [s, e), its scratch at X + xoff
// (schur_tiles(nb) * (e - s) * 32 doubles), its level ranges.
struct SchurJob {
  int64_t s, e, xoff;
  int32_t L0, L1, U0, U1;
};
// S_B -= F_k (L_k U_k)^{-1} E_k for the njobs blocks of a wave (all at once;
// Cpart: njobs * nb * nb doubles), subtracted from S_B in the jobs' order.
cudaError_t schur_wave(int njobs, const SchurJob* jobs, int64_t b0, int64_t nb, const int64_t* prp,
                       const int32_t* pci, const double* pv, const double* F, const double* dinv,
                       const int64_t* pdiag, const int32_t* lev_ptr_lo, const int32_t* lev_rows_lo,
                       const int32_t* lev_ptr_up, const int32_t* lev_rows_up, double* X, double* Cpart, double* SB,
                       cudaStream_t st);
// LU with partial pivoting of the FP64 matrix SB, stored in FP32 (status = 1
// on a zero pivot, 2 if a tensor-core update did not complete).  mode 0:
// blocked with the trailing update on tensor cores, 1: blocked on CUDA cores
// (both with FP64 panels: W holds n x 64 doubles, udiag receives the n
// pivots in FP64), 2: unblocked FP32 (W, udiag unused).
cudaError_t dense_lu_f32(int64_t n, const double* SB, float* LU, int32_t* ipiv, double* W, double* udiag,
                         int* status, int mode, cudaStream_t st);
// Blocked right-looking LU of the FP32 matrix LU in place (dense_lu.cu); FP64
// panels when W and udiag are given.
cudaError_t dense_lu_blocked(int64_t n, float* LU, int32_t* ipiv, double* W, double* udiag, int* status,
                             int tensor_cores, cudaStream_t st);
// Explicit inverse from the LU factors (work: n * 32 * ceil(n / 32) floats).
// mode 0: blocked, block updates on tensor cores; 1: blocked on CUDA cores;
// 2: column tiles swept one row at a time.  status = 2 if a tensor-core
// update did not complete.
cudaError_t dense_lu_inverse(int64_t n, const float* LU, const int32_t* ipiv, const double* udiag, float* Xinv,
                             float* work, int mode, int* status, cudaStream_t st);
cudaError_t dense_inverse_blocked(int64_t n, const float* LU, const int32_t* ipiv, const double* udiag, float* X,
                                  int32_t* perm, int* status, int tensor_cores, cudaStream_t st);
// y = U_k^{-1} L_k^{-1} y on every interior block (in place).
cudaError_t block_lu_solve(int64_t nblocks, const int64_t* bp, const int64_t* prp, const int32_t* pci,
                           const double* F, const double* dinv, const int64_t* pdiag, const int32_t* lev_off_lo,
                           const int32_t* lev_ptr_lo, const int32_t* lev_rows_lo, const int32_t* lev_off_up,
                           const int32_t* lev_ptr_up, const int32_t* lev_rows_up, double* y, cudaStream_t st);
cudaError_t border_gather(int64_t nb, int64_t b0, const int64_t* prp, const int32_t* pci, const double* pv,
                          const double* r, const double* t, double* g, cudaStream_t st);
cudaError_t border_scatter(int64_t b0, const int64_t* prp, const int32_t* pci, const int64_t* pdiag,
                           const double* pv, const double* r, const double* zB, double* w, cudaStream_t st);
// y = A x (A FP32 if A32 != NULL else FP64); residual != 0: y = b - A x.
cudaError_t dense_mv(int64_t n, const float* A32, const double* A64, const double* x, const double* b, double* y,
                     int residual, cudaStream_t st);
cudaError_t axpy(int64_t n, double a, const double* x, double* y, cudaStream_t st);
cudaError_t copy_vec(int64_t n, const double* a, double* b, cudaStream_t st);
int multidot_grid(int64_t n);
// h[i] = V_i^T w (deterministic two-stage), part: nv * multidot_grid(n) doubles.
cudaError_t multidot(int64_t n, int nv, const double* V, int64_t ldv, const double* w, double* part, double* h,
                     cudaStream_t st);
cudaError_t sub_multi(int64_t n, int nv, const double* V, int64_t ldv, const double* h, double* w, cudaStream_t st);
// Modified Gram-Schmidt step: w -= (*hprev) vprev (if vprev), *hout = w^T vcur
// (or w^T w if vcur is NULL); part: multidot_grid(n) doubles.
cudaError_t mgs_step(int64_t n, double* w, const double* vprev, const double* hprev, const double* vcur, double* part,
                     double* hout, cudaStream_t st);
cudaError_t add_multi(int64_t n, int nv, const double* Z, int64_t ldz, const double* y, double* x, cudaStream_t st);
// b = a * s (invert: a / s), s a device scalar.
cudaError_t scale_to(int64_t n, const double* s, int invert, const double* a, double* b, cudaStream_t st);

}  // namespace sdsl
