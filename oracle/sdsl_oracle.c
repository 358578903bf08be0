/*
 * sdsl_oracle.c -- plain, slow, single-threaded FP64 reference of the
 * SDSL-Solver hot path (arXiv 2604.23979).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or helper with the CUDA
 * path.  It is compiled with -O2 -ffp-contract=off so that every a*b+c is two
 * roundings unless fma() is written out.
 *
 * Each routine follows one passage of the paper:
 *   or_normal_*        normal-equation matrix S = B D^{-1} B^T of Eq. (schur)
 *                      (here A diag(theta) A^T + rho I, the IPM scaling
 *                      D^{-1} = diag(theta)), with a fixed rounding order;
 *   or_augmented       the augmented matrix of Eq. (augmented), in bordered
 *                      block-diagonal (BBD) order, Sec. 2.4;
 *   or_filter_correct  numerics-based filtering, Eq. (filter) / Algorithm 2,
 *                      then diagonal correction, Eq. (diagcorr) / Algorithm 3;
 *   or_levels          level sets of the triangular solves of Sec. 2.3
 *                      ("solve the precondition system");
 *   or_ic0 / or_ilu0   per-block IC(0) / ILU(0), Sec. 2.3 (third step) and
 *                      the factor options of Sec. 3.1;
 *   or_pcg             right-preconditioned Block-Jacobi CG (Sec. 2.2-2.3);
 *   or_bbd_* / or_gmres  BBD Schur complement, block solve (Sec. 2.4) and
 *                      right-preconditioned restarted GMRES (Sec. 2.2);
 *   or_bicgstab        right-preconditioned BiCGSTAB, the method paired with
 *                      Block Jacobi in Sec. 4.3 (van der Vorst 1992);
 *   or_gcr             restarted right-preconditioned GCR(m), the "IGCR(m)"
 *                      paired with BBD in Sec. 4.3 (Eisenstat et al. 1983).
 *
 * Conventions: CSR with int64 row pointers, int32 sorted column indices,
 * double values.  Blocks are contiguous index ranges block_ptr[b] ..
 * block_ptr[b+1].  All routines return 0 on success.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Independent loops (rows of a product, blocks of a block-diagonal
 * operation) run in parallel when the file is built with OpenMP; every
 * reduction (dot products, norms, sums) is computed by one thread in a
 * fixed order, and each parallel iteration writes only its own rows, so the
 * results are the same bits with or without threads. */
#if defined(_OPENMP)
#include <omp.h>
#define OR_PARALLEL_ROWS _Pragma("omp parallel for schedule(static)")
#define OR_PARALLEL_BLOCKS _Pragma("omp parallel for schedule(dynamic, 1)")
int or_threads(void) { return omp_get_max_threads(); }
#else
#define OR_PARALLEL_ROWS
#define OR_PARALLEL_BLOCKS
int or_threads(void) { return 1; }
#endif

#define OR_OK 0
#define OR_BREAKDOWN 4
#define OR_NOT_CONVERGED 5
#define OR_ARG 1
#define OR_OOM 2

/* ------------------------------------------------------------------ */
/* small utilities                                                     */
/* ------------------------------------------------------------------ */

/* position of column c in row i of a sorted CSR, or -1 */
static int64_t find_in_row(const int64_t* rp, const int32_t* ci, int64_t i, int32_t c) {
  int64_t lo = rp[i], hi = rp[i + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (ci[mid] == c) return mid;
    if (ci[mid] < c) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static int64_t block_of(int64_t nblocks, const int64_t* block_ptr, int64_t i) {
  /* largest b with block_ptr[b] <= i; nblocks if i is past the last block */
  int64_t lo = 0, hi = nblocks;
  if (i >= block_ptr[nblocks]) return nblocks;
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) / 2;
    if (block_ptr[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

/* ------------------------------------------------------------------ */
/* transpose                                                           */
/* ------------------------------------------------------------------ */

/* CSR of A^T (n x m) from CSR of A (m x n); rows of the result sorted. */
void or_transpose(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                  int64_t* trp, int32_t* tci, double* tv) {
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  memset(trp, 0, sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t i = 0; i < m; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) trp[ci[p] + 1]++;
  for (int64_t j = 0; j < n; ++j) trp[j + 1] += trp[j];
  memcpy(next, trp, sizeof(int64_t) * (size_t)(n + 1));
  /* rows visited in ascending order, so every column list comes out sorted */
  for (int64_t i = 0; i < m; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t q = next[ci[p]]++;
      tci[q] = (int32_t)i;
      if (tv) tv[q] = v[p];
    }
  free(next);
}

/* ------------------------------------------------------------------ */
/* Eq. (schur): S = A diag(theta) A^T + rho I                          */
/* ------------------------------------------------------------------ */

/* Pattern of S.  Row i holds i itself and every row j that shares a column
 * of A with row i (the structural product; cancellation is not detected).
 * Call with sci == NULL to fill srp (counts + prefix) only. */
int64_t or_normal_pattern(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci,
                          const int64_t* trp, const int32_t* tci, int64_t* srp, int32_t* sci) {
  (void)n;
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  for (int64_t i = 0; i < m; ++i) mark[i] = -1;
  if (sci == NULL) srp[0] = 0;
  for (int64_t i = 0; i < m; ++i) {
    int64_t cnt = 0;
    mark[i] = (int32_t)i;
    list[cnt++] = (int32_t)i;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int32_t k = ci[p];
      for (int64_t q = trp[k]; q < trp[k + 1]; ++q) {
        int32_t j = tci[q];
        if (mark[j] != (int32_t)i) { mark[j] = (int32_t)i; list[cnt++] = j; }
      }
    }
    if (sci == NULL) {
      srp[i + 1] = srp[i] + cnt;
    } else {
      qsort(list, (size_t)cnt, sizeof(int32_t), cmp_i32);
      memcpy(sci + srp[i], list, sizeof(int32_t) * (size_t)cnt);
    }
  }
  free(mark);
  free(list);
  return srp[m];
}

/* Values of S on its pattern.  Fixed rounding (so that the pattern after
 * filtering can be compared bit for bit): for an entry (i, j) let h = max(i,j)
 * and l = min(i,j); then
 *     S_ij = sum over k in cols(h) & cols(l), k ascending, of
 *            acc = fma(fl(a_hk * theta_k), a_lk, acc),  acc starting at +0,
 * and S_ii = fl(acc + rho).  The h/l rule makes S exactly symmetric. */
void or_normal_values(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                      const double* theta, double rho, const int64_t* srp, const int32_t* sci,
                      double* sv) {
  (void)n;
  OR_PARALLEL_ROWS
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t s = srp[i]; s < srp[i + 1]; ++s) {
      int64_t j = sci[s];
      int64_t h = i > j ? i : j, l = i > j ? j : i;
      double acc = 0.0;
      int64_t ph = rp[h], pl = rp[l];
      while (ph < rp[h + 1] && pl < rp[l + 1]) { /* sorted merge of the two rows */
        if (ci[ph] < ci[pl]) ++ph;
        else if (ci[ph] > ci[pl]) ++pl;
        else {
          double t = v[ph] * theta[ci[ph]];
          acc = fma(t, v[pl], acc);
          ++ph; ++pl;
        }
      }
      if (i == j) acc = acc + rho;
      sv[s] = acc;
    }
  }
}

/* ------------------------------------------------------------------ */
/* Eq. (augmented) in BBD order (Sec. 2.4)                             */
/* ------------------------------------------------------------------ */

/* Position of every unknown of K = [[-diag(1/theta), A^T], [A, rho I]]
 * (x_j = index j, lambda_i = index n+i) in the bordered block-diagonal order:
 * for each block k the columns of A's block k (x_k) then its rows
 * (lambda_k), and finally the linking rows of A (the border).
 * Outputs pos[n+m] (old -> new) and the block pointer over the new order. */
void or_bbd_order(int64_t m, int64_t n, int64_t nblocks, const int64_t* row_block_ptr,
                  const int64_t* col_block_ptr, int64_t* pos, int64_t* kblock_ptr) {
  int64_t at = 0;
  for (int64_t k = 0; k < nblocks; ++k) {
    kblock_ptr[k] = at;
    for (int64_t j = col_block_ptr[k]; j < col_block_ptr[k + 1]; ++j) pos[j] = at++;
    for (int64_t i = row_block_ptr[k]; i < row_block_ptr[k + 1]; ++i) pos[n + i] = at++;
  }
  kblock_ptr[nblocks] = at;
  for (int64_t i = row_block_ptr[nblocks]; i < m; ++i) pos[n + i] = at++;
}

/* Assemble K in the order given by pos.  Call with kci == NULL to fill
 * krp only.  Diagonal of x_j is fl(-1/theta_j), of lambda_i is rho. */
int64_t or_augmented(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                     const int64_t* trp, const int32_t* tci, const double* tv, const double* theta,
                     double rho, const int64_t* pos, int64_t* krp, int32_t* kci, double* kv) {
  int64_t N = n + m;
  int64_t* inv = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  for (int64_t u = 0; u < N; ++u) inv[pos[u]] = u;
  if (kci == NULL) krp[0] = 0;
  int32_t* cbuf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  double* vbuf = (double*)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
  for (int64_t r = 0; r < N; ++r) {
    int64_t u = inv[r], cnt = 0;
    if (u < n) { /* x_u: diagonal, then A^T row u = column u of A */
      cbuf[cnt] = (int32_t)pos[u]; vbuf[cnt++] = -1.0 / theta[u];
      for (int64_t q = trp[u]; q < trp[u + 1]; ++q) { cbuf[cnt] = (int32_t)pos[n + tci[q]]; vbuf[cnt++] = tv[q]; }
    } else {     /* lambda_i: row i of A, then diagonal rho */
      int64_t i = u - n;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) { cbuf[cnt] = (int32_t)pos[ci[p]]; vbuf[cnt++] = v[p]; }
      cbuf[cnt] = (int32_t)pos[u]; vbuf[cnt++] = rho;
    }
    if (kci == NULL) { krp[r + 1] = krp[r] + cnt; continue; }
    /* insertion sort by new column (rows are short) */
    for (int64_t a = 0; a < cnt; ++a) ord[a] = a;
    for (int64_t a = 1; a < cnt; ++a) {
      int64_t t = ord[a], b = a - 1;
      while (b >= 0 && cbuf[ord[b]] > cbuf[t]) { ord[b + 1] = ord[b]; --b; }
      ord[b + 1] = t;
    }
    for (int64_t a = 0; a < cnt; ++a) { kci[krp[r] + a] = cbuf[ord[a]]; kv[krp[r] + a] = vbuf[ord[a]]; }
  }
  free(inv); free(cbuf); free(vbuf); free(ord);
  return krp[N];
}

/* ------------------------------------------------------------------ */
/* Eq. (filter) + Eq. (diagcorr): build the preconditioner matrix P    */
/* ------------------------------------------------------------------ */

/* P from matrix S (n x n):
 *   - scope: if whole == 0 only entries whose row and column lie in the same
 *     block (block_ptr, nblocks) enter P (Block Jacobi, Sec. 2.3); if
 *     whole == 1 every entry does (BBD keeps the border, Sec. 2.4);
 *   - filter (Eq. filter, Algorithm 2): an off-diagonal s_ij is dropped when
 *     |s_ij| < fl(tau*|s_ii|) and |s_ij| < fl(tau*|s_jj|), strict "<";
 *     every diagonal entry is kept (a missing one is inserted as 0);
 *   - correction (Eq. diagcorr, Algorithm 3 step 3): p_ii = fl(s_ii +
 *     delta*sign(s_ii)) with sign(0) = +1, on P only.
 * Call with pci == NULL to fill prp only. */
int64_t or_filter_correct(int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                          int64_t nblocks, const int64_t* block_ptr, int whole, double tau,
                          double delta, int64_t* prp, int32_t* pci, double* pv) {
  double* d = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  for (int64_t i = 0; i < n; ++i) {
    int64_t p = find_in_row(rp, ci, i, (int32_t)i);
    d[i] = p >= 0 ? v[p] : 0.0;
  }
  if (pci == NULL) prp[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t bi = block_of(nblocks, block_ptr, i);
    int64_t cnt = 0, at = pci ? prp[i] : 0;
    int have_diag = 0;
    double ti = tau * fabs(d[i]);
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      if (!whole && block_of(nblocks, block_ptr, j) != bi) continue;
      if (j != i) {
        double a = fabs(v[p]);
        double tj = tau * fabs(d[j]);
        if (a < ti && a < tj) continue; /* dropped */
      }
      if (j > i && !have_diag) { /* missing diagonal goes before the first j > i */
        if (pci) { pci[at + cnt] = (int32_t)i; pv[at + cnt] = 0.0 + (delta); }
        ++cnt; have_diag = 1;
      }
      if (pci) {
        pci[at + cnt] = (int32_t)j;
        if (j == i) {
          double sg = v[p] < 0.0 ? -1.0 : 1.0;
          pv[at + cnt] = v[p] + delta * sg;
        } else {
          pv[at + cnt] = v[p];
        }
      }
      if (j == i) have_diag = 1;
      ++cnt;
    }
    if (!have_diag) {
      if (pci) { pci[at + cnt] = (int32_t)i; pv[at + cnt] = 0.0 + delta; }
      ++cnt;
    }
    if (pci == NULL) prp[i + 1] = prp[i] + cnt;
  }
  free(d);
  return prp[n];
}

/* ------------------------------------------------------------------ */
/* level sets of the block triangular solves (Sec. 2.3)                */
/* ------------------------------------------------------------------ */

/* For every row i of a block: lower level = 0 if row i has no in-block
 * entry left of the diagonal, else 1 + max lower level of those columns j < i;
 * upper level = 0 if no in-block entry right of the diagonal, else
 * 1 + max upper level over those j > i (evaluated from the block's last row
 * backwards).  Rows outside every block get level -1. */
void or_levels(int64_t n, const int64_t* rp, const int32_t* ci, int64_t nblocks,
               const int64_t* block_ptr, int32_t* lev_lo, int32_t* lev_up) {
  for (int64_t i = 0; i < n; ++i) { lev_lo[i] = -1; lev_up[i] = -1; }
  OR_PARALLEL_BLOCKS
  for (int64_t b = 0; b < nblocks; ++b) {
    int64_t s = block_ptr[b], e = block_ptr[b + 1];
    for (int64_t i = s; i < e; ++i) {
      int32_t best = -1;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int64_t j = ci[p];
        if (j >= s && j < i && lev_lo[j] > best) best = lev_lo[j];
      }
      lev_lo[i] = best + 1;
    }
    for (int64_t i = e - 1; i >= s; --i) {
      int32_t best = -1;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int64_t j = ci[p];
        if (j > i && j < e && lev_up[j] > best) best = lev_up[j];
      }
      lev_up[i] = best + 1;
    }
  }
}

/* Level lists: for each block, its levels in order, the rows of each level
 * ascending.  nlev[b] = number of levels of block b; level_ptr has
 * sum(nlev)+1 entries (offsets into level_rows, which lists every block row
 * once, block by block).  Call with level_ptr == NULL to fill nlev only. */
void or_level_lists(int64_t nblocks, const int64_t* block_ptr, const int32_t* lev, int32_t* nlev,
                    int64_t* level_ptr, int32_t* level_rows) {
  int64_t L = 0, at = block_ptr[0];
  if (level_ptr) level_ptr[0] = block_ptr[0];
  for (int64_t b = 0; b < nblocks; ++b) {
    int32_t mx = -1;
    for (int64_t i = block_ptr[b]; i < block_ptr[b + 1]; ++i) if (lev[i] > mx) mx = lev[i];
    nlev[b] = mx + 1;
    if (!level_ptr) continue;
    for (int32_t l = 0; l <= mx; ++l) {
      for (int64_t i = block_ptr[b]; i < block_ptr[b + 1]; ++i)
        if (lev[i] == l) level_rows[at++ - block_ptr[0]] = (int32_t)i;
      level_ptr[++L] = at;
    }
  }
}

/* ------------------------------------------------------------------ */
/* IC(0) per block (Sec. 2.3, third step)                              */
/* ------------------------------------------------------------------ */


/* diagonal of P for shift alpha: p_ii if alpha == 0, else fl(p_ii + fl(alpha*p_ii)) */
static double shifted(double pii, double alpha) { return alpha == 0.0 ? pii : pii + alpha * pii; }

/* One block of IC(0), row by row: for row i and every k < i of its pattern
 * (ascending), l_ik = (p_ik - sum_{j<k, (i,j),(k,j) in pattern} l_ij l_kj) / l_kk,
 * then l_ii = sqrt(p_ii - sum_{j<i} l_ij^2).  A pivot that is not > 0 or not
 * finite is a breakdown.  F has the layout of P; only in-block positions with
 * j <= i are written. */
static int ic0_block(const int64_t* rp, const int32_t* ci, const double* pv, int64_t s, int64_t e,
                     double alpha, double* F) {
  for (int64_t i = s; i < e; ++i) {
    int64_t dpos = -1;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t k = ci[p];
      if (k < s) continue;
      if (k >= i) { if (k == i) dpos = p; break; }
      double acc = pv[p];
      /* sum over j < k in row i that also appear in row k */
      for (int64_t q = rp[i]; q < p; ++q) {
        int64_t j = ci[q];
        if (j < s) continue;
        int64_t kq = find_in_row(rp, ci, k, (int32_t)j);
        if (kq >= 0) acc = acc - F[q] * F[kq];
      }
      int64_t kd = find_in_row(rp, ci, k, (int32_t)k);
      F[p] = acc / F[kd];
    }
    if (dpos < 0) return 1;
    double dsum = shifted(pv[dpos], alpha);
    for (int64_t q = rp[i]; q < dpos; ++q) {
      if (ci[q] < s) continue;
      dsum = dsum - F[q] * F[q];
    }
    if (!(dsum > 0.0) || !isfinite(dsum)) return 1;
    F[dpos] = sqrt(dsum);
  }
  return 0;
}

/* IC(0) of every block of P with the shift-retry rule: the block is factored
 * with diagonal p_ii + alpha*p_ii for alpha = shifts[0], shifts[1], ... in
 * turn until no pivot breaks down (Manteuffel's shifted incomplete Cholesky;
 * shifts[0] is normally 0, i.e. the unshifted factor first);
 * alpha_used[b] records the shift (-1 if every shift failed). */
int or_ic0(int64_t n, const int64_t* rp, const int32_t* ci, const double* pv, int64_t nblocks,
           const int64_t* block_ptr, const double* shifts, int nshifts, double* F, double* alpha_used) {
  (void)n;
  int status = OR_OK;
  OR_PARALLEL_BLOCKS
  for (int64_t b = 0; b < nblocks; ++b) {
    alpha_used[b] = -1.0;
    for (int t = 0; t < nshifts; ++t) {
      if (ic0_block(rp, ci, pv, block_ptr[b], block_ptr[b + 1], shifts[t], F) == 0) {
        alpha_used[b] = shifts[t];
        break;
      }
    }
  }
  for (int64_t b = 0; b < nblocks; ++b)
    if (alpha_used[b] < 0) status = OR_BREAKDOWN;
  return status;
}

/* ------------------------------------------------------------------ */
/* ILU(0) per block (Sec. 3.1 factor options; BBD blocks, Sec. 2.4)    */
/* ------------------------------------------------------------------ */

/* IKJ ILU(0) restricted to the in-block pattern: for row i, for each k < i
 * of the pattern (ascending), l_ik = w_ik / u_kk, then w_ij -= l_ik u_kj for
 * every j > k present in both row i and row k.  L is unit lower (its
 * multipliers stored at j < i), U upper (j >= i).  A zero or non-finite pivot
 * is a breakdown. */
static int ilu0_block(const int64_t* rp, const int32_t* ci, const double* pv, int64_t s, int64_t e,
                      double alpha, double* F) {
  for (int64_t i = s; i < e; ++i) {
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      if (j >= s && j < e) F[p] = (j == i) ? shifted(pv[p], alpha) : pv[p];
    }
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t k = ci[p];
      if (k < s) continue;
      if (k >= i) break;
      int64_t kd = find_in_row(rp, ci, k, (int32_t)k);
      F[p] = F[p] / F[kd];
      for (int64_t q = p + 1; q < rp[i + 1]; ++q) {
        int64_t j = ci[q];
        if (j >= e) break;
        int64_t kq = find_in_row(rp, ci, k, (int32_t)j);
        if (kq >= 0) F[q] = F[q] - F[p] * F[kq];
      }
    }
    int64_t dpos = find_in_row(rp, ci, i, (int32_t)i);
    if (dpos < 0) return 1;
    if (F[dpos] == 0.0 || !isfinite(F[dpos])) return 1;
  }
  return 0;
}

int or_ilu0(int64_t n, const int64_t* rp, const int32_t* ci, const double* pv, int64_t nblocks,
            const int64_t* block_ptr, const double* shifts, int nshifts, double* F, double* alpha_used) {
  (void)n;
  int status = OR_OK;
  OR_PARALLEL_BLOCKS
  for (int64_t b = 0; b < nblocks; ++b) {
    alpha_used[b] = -1.0;
    for (int t = 0; t < nshifts; ++t) {
      if (ilu0_block(rp, ci, pv, block_ptr[b], block_ptr[b + 1], shifts[t], F) == 0) {
        alpha_used[b] = shifts[t];
        break;
      }
    }
  }
  for (int64_t b = 0; b < nblocks; ++b)
    if (alpha_used[b] < 0) status = OR_BREAKDOWN;
  return status;
}

/* ------------------------------------------------------------------ */
/* block triangular solves                                             */
/* ------------------------------------------------------------------ */

/* z = (L L^T)^{-1} r on every block (IC(0) factor in F, layout of P). */
void or_ic0_apply(int64_t n, const int64_t* rp, const int32_t* ci, const double* F, int64_t nblocks,
                  const int64_t* block_ptr, const double* r, double* z) {
  (void)n;
  OR_PARALLEL_BLOCKS
  for (int64_t b = 0; b < nblocks; ++b) {
    int64_t s = block_ptr[b], e = block_ptr[b + 1];
    /* forward: L y = r (y kept in z) */
    for (int64_t i = s; i < e; ++i) {
      double acc = r[i];
      int64_t dpos = -1;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        int64_t j = ci[p];
        if (j < s) continue;
        if (j >= i) { dpos = p; break; }
        acc = acc - F[p] * z[j];
      }
      z[i] = acc / F[dpos];
    }
    /* backward: L^T z = y, column-oriented over the rows of L */
    for (int64_t i = e - 1; i >= s; --i) {
      int64_t dpos = find_in_row(rp, ci, i, (int32_t)i);
      z[i] = z[i] / F[dpos];
      for (int64_t p = rp[i]; p < dpos; ++p) {
        int64_t j = ci[p];
        if (j < s) continue;
        z[j] = z[j] - F[p] * z[i];
      }
    }
  }
}

/* y_k = L_k^{-1} r_k (unit lower) on block [s, e) of an ILU(0) factor */
static void ilu0_lower(const int64_t* rp, const int32_t* ci, const double* F, int64_t s, int64_t e,
                       const double* r, double* y) {
  for (int64_t i = s; i < e; ++i) {
    double acc = r[i];
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      if (j < s) continue;
      if (j >= i) break;
      acc = acc - F[p] * y[j];
    }
    y[i] = acc;
  }
}

/* z_k = U_k^{-1} y_k on block [s, e) */
static void ilu0_upper(const int64_t* rp, const int32_t* ci, const double* F, int64_t s, int64_t e,
                       const double* y, double* z) {
  for (int64_t i = e - 1; i >= s; --i) {
    double acc = y[i];
    int64_t dpos = -1;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t j = ci[p];
      if (j < i) continue;
      if (j >= e) break;
      if (j == i) { dpos = p; continue; }
      acc = acc - F[p] * z[j];
    }
    z[i] = acc / F[dpos];
  }
}

/* z = (L U)^{-1} r on every block (Block Jacobi with ILU(0)). */
void or_ilu0_apply(int64_t n, const int64_t* rp, const int32_t* ci, const double* F, int64_t nblocks,
                   const int64_t* block_ptr, const double* r, double* z) {
  double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  OR_PARALLEL_BLOCKS
  for (int64_t b = 0; b < nblocks; ++b) {
    ilu0_lower(rp, ci, F, block_ptr[b], block_ptr[b + 1], r, y);
    ilu0_upper(rp, ci, F, block_ptr[b], block_ptr[b + 1], y, z);
  }
  free(y);
}

/* ------------------------------------------------------------------ */
/* BLAS-1 and SpMV                                                     */
/* ------------------------------------------------------------------ */

void or_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* x, double* y) {
  OR_PARALLEL_ROWS
  for (int64_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) acc = acc + v[p] * x[ci[p]];
    y[i] = acc;
  }
}

/* Inner product by pairwise (cascade) summation: halves summed recursively,
 * runs of at most 32 products in index order.  The paper does not fix the
 * summation order; this one keeps the rounding-error bound of a length-n sum
 * at O(eps log n) instead of the O(n eps) of one serial pass (Higham,
 * "The accuracy of floating point summation", 1993), so the reference
 * iteration counts of 10^5-10^6-long Krylov vectors are not set by
 * summation error.  Deterministic: the split depends on n only. */
static double dot_pairwise(const double* a, const double* b, int64_t n) {
  if (n <= 32) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
    return s;
  }
  const int64_t h = n / 2;
  return dot_pairwise(a, b, h) + dot_pairwise(a + h, b + h, n - h);
}

static double dot(int64_t n, const double* a, const double* b) { return dot_pairwise(a, b, n); }

static double nrm2(int64_t n, const double* a) { return sqrt(dot(n, a, a)); }

/* ------------------------------------------------------------------ */
/* BBD: Schur complement, dense LU, block solve (Sec. 2.4)             */
/* ------------------------------------------------------------------ */

/* Dense LU with partial pivoting, row-major nb x nb, in place.  The pivot is
 * the entry of largest magnitude in the column, the lowest row on ties. */
int or_dense_lu(int64_t nb, double* a, int32_t* ipiv) {
  for (int64_t k = 0; k < nb; ++k) {
    int64_t piv = k;
    double best = fabs(a[k * nb + k]);
    for (int64_t i = k + 1; i < nb; ++i)
      if (fabs(a[i * nb + k]) > best) { best = fabs(a[i * nb + k]); piv = i; }
    ipiv[k] = (int32_t)piv;
    if (best == 0.0 || !isfinite(best)) return OR_BREAKDOWN;
    if (piv != k)
      for (int64_t j = 0; j < nb; ++j) { double t = a[k * nb + j]; a[k * nb + j] = a[piv * nb + j]; a[piv * nb + j] = t; }
    for (int64_t i = k + 1; i < nb; ++i) {
      double l = a[i * nb + k] / a[k * nb + k];
      a[i * nb + k] = l;
      for (int64_t j = k + 1; j < nb; ++j) a[i * nb + j] = a[i * nb + j] - l * a[k * nb + j];
    }
  }
  return OR_OK;
}

void or_dense_lu_solve(int64_t nb, const double* lu, const int32_t* ipiv, double* x) {
  for (int64_t k = 0; k < nb; ++k) { int64_t p = ipiv[k]; if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; } }
  for (int64_t i = 0; i < nb; ++i) { double acc = x[i]; for (int64_t j = 0; j < i; ++j) acc = acc - lu[i * nb + j] * x[j]; x[i] = acc; }
  for (int64_t i = nb - 1; i >= 0; --i) {
    double acc = x[i];
    for (int64_t j = i + 1; j < nb; ++j) acc = acc - lu[i * nb + j] * x[j];
    x[i] = acc / lu[i * nb + i];
  }
}

/* Schur complement of the BBD preconditioner (Sec. 2.4, third step):
 *   S_B = C - sum_k F_k (L_k U_k)^{-1} E_k,
 * with E_k = P[block k rows, border cols], F_k = P[border rows, block k cols],
 * C = P[border, border] and L_k U_k the ILU(0) factor of block k.  The border
 * is rows/cols block_ptr[nblocks] .. n-1.  SB is row-major nb x nb. */
void or_bbd_schur(int64_t n, const int64_t* rp, const int32_t* ci, const double* pv, const double* F,
                  int64_t nblocks, const int64_t* block_ptr, double* SB) {
  int64_t b0 = block_ptr[nblocks], nb = n - b0;
  for (int64_t i = 0; i < nb * nb; ++i) SB[i] = 0.0;
  for (int64_t r = 0; r < nb; ++r)
    for (int64_t p = rp[b0 + r]; p < rp[b0 + r + 1]; ++p)
      if (ci[p] >= b0) SB[r * nb + (ci[p] - b0)] = pv[p];
  double* e = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t k = 0; k < nblocks; ++k) {
    int64_t s = block_ptr[k], t = block_ptr[k + 1];
    for (int64_t c = 0; c < nb; ++c) {
      int any = 0;
      for (int64_t i = s; i < t; ++i) {
        int64_t p = find_in_row(rp, ci, i, (int32_t)(b0 + c));
        e[i] = p >= 0 ? pv[p] : 0.0;
        any |= (p >= 0);
      }
      if (!any) continue;
      ilu0_lower(rp, ci, F, s, t, e, w);
      ilu0_upper(rp, ci, F, s, t, w, y);
      for (int64_t r = 0; r < nb; ++r) {
        double acc = 0.0;
        for (int64_t p = rp[b0 + r]; p < rp[b0 + r + 1]; ++p) {
          int64_t j = ci[p];
          if (j >= s && j < t) acc = acc + pv[p] * y[j];
        }
        SB[r * nb + c] = SB[r * nb + c] - acc;
      }
    }
  }
  free(e); free(y); free(w);
}

/* z = M^{-1} r for the BBD preconditioner (Sec. 2.4, fourth step):
 *   y_k = L_k^{-1} r_k;  g = r_B - sum_k F_k U_k^{-1} y_k;  z_B = S_B^{-1} g;
 *   z_k = U_k^{-1} (y_k - L_k^{-1} E_k z_B). */
void or_bbd_apply(int64_t n, const int64_t* rp, const int32_t* ci, const double* pv, const double* F,
                  int64_t nblocks, const int64_t* block_ptr, const double* lu, const int32_t* ipiv,
                  const double* r, double* z) {
  int64_t b0 = block_ptr[nblocks], nb = n - b0;
  double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* t = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* g = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
  for (int64_t k = 0; k < nblocks; ++k) ilu0_lower(rp, ci, F, block_ptr[k], block_ptr[k + 1], r, y);
  for (int64_t k = 0; k < nblocks; ++k) ilu0_upper(rp, ci, F, block_ptr[k], block_ptr[k + 1], y, t);
  for (int64_t r0 = 0; r0 < nb; ++r0) {
    double acc = r[b0 + r0];
    for (int64_t p = rp[b0 + r0]; p < rp[b0 + r0 + 1]; ++p)
      if (ci[p] < b0) acc = acc - pv[p] * t[ci[p]];
    g[r0] = acc;
  }
  or_dense_lu_solve(nb, lu, ipiv, g);
  for (int64_t c = 0; c < nb; ++c) z[b0 + c] = g[c];
  /* y_k - L_k^{-1} E_k z_B = L_k^{-1} (r_k - E_k z_B) */
  for (int64_t i = 0; i < b0; ++i) {
    double acc = r[i];
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] >= b0) acc = acc - pv[p] * g[ci[p] - b0];
    t[i] = acc;
  }
  for (int64_t k = 0; k < nblocks; ++k) {
    ilu0_lower(rp, ci, F, block_ptr[k], block_ptr[k + 1], t, y);
    ilu0_upper(rp, ci, F, block_ptr[k], block_ptr[k + 1], y, z);
  }
  free(y); free(t); free(g);
}

/* ------------------------------------------------------------------ */
/* Krylov solvers (Sec. 2.2; tolerance 1e-8 as in Sec. 4)              */
/* ------------------------------------------------------------------ */

typedef struct {
  int kind; /* 0 none, 1 BJ IC(0), 2 BJ ILU(0), 3 BBD */
  int64_t n;
  const int64_t* rp; const int32_t* ci; const double* pv; const double* F;
  int64_t nblocks; const int64_t* block_ptr;
  const double* lu; const int32_t* ipiv;
} or_precond;

static void precond_apply(const or_precond* M, const double* r, double* z) {
  switch (M->kind) {
    case 1: or_ic0_apply(M->n, M->rp, M->ci, M->F, M->nblocks, M->block_ptr, r, z); break;
    case 2: or_ilu0_apply(M->n, M->rp, M->ci, M->F, M->nblocks, M->block_ptr, r, z); break;
    case 3: or_bbd_apply(M->n, M->rp, M->ci, M->pv, M->F, M->nblocks, M->block_ptr, M->lu, M->ipiv, r, z); break;
    default: memcpy(z, r, sizeof(double) * (size_t)M->n);
  }
}

/* Preconditioned CG.  x holds x0 on entry (zeros for a cold start) and the
 * iterate on exit.  The count is the number of products q = S p.  When the
 * recurrence residual reaches rtol*||b|| the true residual ||b - S x|| is
 * recomputed; if it has not reached the tolerance the iteration restarts from
 * r = b - S x (new direction p = M^{-1} r).  out[0] = true relative residual,
 * out[1] = recurrence relative residual. */
int or_pcg(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const or_precond* M,
           const double* b, double* x, double rtol, int64_t maxit, int64_t* iters, double* out) {
  double *r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *q = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int status = OR_NOT_CONVERGED;
  int64_t it = 0;
  double bnorm = nrm2(n, b), rnorm = 0.0, tnorm = 0.0;
  double tol = rtol * bnorm;
  or_spmv(n, rp, ci, v, x, q);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
  rnorm = nrm2(n, r);
  tnorm = rnorm;
  if (bnorm == 0.0) { for (int64_t i = 0; i < n; ++i) x[i] = 0.0; rnorm = tnorm = 0.0; status = OR_OK; goto done; }
  if (rnorm <= tol) { status = OR_OK; goto done; }
  precond_apply(M, r, z);
  memcpy(p, z, sizeof(double) * (size_t)n);
  double rho = dot(n, r, z);
  while (it < maxit) {
    or_spmv(n, rp, ci, v, p, q);
    ++it;
    double pq = dot(n, p, q);
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rho)) { status = OR_BREAKDOWN; break; }
    double alpha = rho / pq;
    for (int64_t i = 0; i < n; ++i) { x[i] = x[i] + alpha * p[i]; r[i] = r[i] - alpha * q[i]; }
    rnorm = nrm2(n, r);
    if (rnorm <= tol) {
      or_spmv(n, rp, ci, v, x, q);
      for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
      tnorm = nrm2(n, q);
      if (tnorm <= tol) { status = OR_OK; break; }
      memcpy(r, q, sizeof(double) * (size_t)n);
      rnorm = tnorm;
      precond_apply(M, r, z);
      memcpy(p, z, sizeof(double) * (size_t)n);
      rho = dot(n, r, z);
      continue;
    }
    precond_apply(M, r, z);
    double rho_new = dot(n, r, z);
    double beta = rho_new / rho;
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rho = rho_new;
  }
  if (status != OR_OK) {
    or_spmv(n, rp, ci, v, x, q);
    for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
    tnorm = nrm2(n, q);
  }
done:
  *iters = it;
  out[0] = bnorm > 0.0 ? tnorm / bnorm : 0.0;
  out[1] = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  free(r); free(z); free(p); free(q);
  return status;
}

/* Right-preconditioned restarted GMRES(m) with modified Gram-Schmidt and
 * Givens rotations: solves K M^{-1} u = b, x = M^{-1} u, keeping the
 * preconditioned directions Z_j = M^{-1} V_j.  The count is the number of
 * Arnoldi steps (products K z), summed over restarts.  Convergence is tested
 * on |g_{j+1}| <= rtol*||b|| and confirmed with the true residual at the end
 * of each cycle. */
int or_gmres(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const or_precond* M,
             const double* b, double* x, double rtol, int64_t maxit, int64_t restart, int64_t* iters,
             double* out) {
  int64_t m = restart;
  double* V = (double*)malloc(sizeof(double) * (size_t)(n * (m + 1) > 0 ? n * (m + 1) : 1));
  double* Z = (double*)malloc(sizeof(double) * (size_t)(n * m > 0 ? n * m : 1));
  double* H = (double*)calloc((size_t)((m + 1) * m), sizeof(double));
  double* cs = (double*)malloc(sizeof(double) * (size_t)m);
  double* sn = (double*)malloc(sizeof(double) * (size_t)m);
  double* g = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* yv = (double*)malloc(sizeof(double) * (size_t)m);
  double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int status = OR_NOT_CONVERGED;
  int64_t it = 0;
  double bnorm = nrm2(n, b), tol = rtol * bnorm, tnorm = 0.0, gres = 0.0;
  if (bnorm == 0.0) { for (int64_t i = 0; i < n; ++i) x[i] = 0.0; status = OR_OK; goto done; }
  for (;;) {
    or_spmv(n, rp, ci, v, x, w);
    for (int64_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
    double beta = nrm2(n, w);
    tnorm = beta;
    gres = beta;
    if (beta <= tol) { status = OR_OK; break; }
    if (it >= maxit) break;
    for (int64_t i = 0; i < n; ++i) V[i] = w[i] / beta;
    for (int64_t i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    int64_t jend = 0;
    for (int64_t j = 0; j < m; ++j) {
      precond_apply(M, V + j * n, Z + j * n);
      or_spmv(n, rp, ci, v, Z + j * n, w);
      ++it;
      for (int64_t i = 0; i <= j; ++i) {
        double h = dot(n, w, V + i * n);
        H[i * m + j] = h;
        for (int64_t l = 0; l < n; ++l) w[l] = w[l] - h * V[i * n + l];
      }
      double hn = nrm2(n, w);
      H[(j + 1) * m + j] = hn;
      if (hn != 0.0)
        for (int64_t l = 0; l < n; ++l) V[(j + 1) * n + l] = w[l] / hn;
      for (int64_t i = 0; i < j; ++i) {
        double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      double a = H[j * m + j], c = H[(j + 1) * m + j];
      double rr = hypot(a, c);
      cs[j] = rr == 0.0 ? 1.0 : a / rr;
      sn[j] = rr == 0.0 ? 0.0 : c / rr;
      H[j * m + j] = rr;
      H[(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      gres = fabs(g[j + 1]);
      jend = j + 1;
      if (gres <= tol || it >= maxit || hn == 0.0) break;
    }
    for (int64_t i = jend - 1; i >= 0; --i) {
      double acc = g[i];
      for (int64_t l = i + 1; l < jend; ++l) acc = acc - H[i * m + l] * yv[l];
      yv[i] = acc / H[i * m + i];
    }
    for (int64_t i = 0; i < jend; ++i)
      for (int64_t l = 0; l < n; ++l) x[l] = x[l] + yv[i] * Z[i * n + l];
    or_spmv(n, rp, ci, v, x, w);
    for (int64_t i = 0; i < n; ++i) w[i] = b[i] - w[i];
    tnorm = nrm2(n, w);
    if (tnorm <= tol) { status = OR_OK; break; }
    if (it >= maxit) break;
  }
done:
  *iters = it;
  out[0] = bnorm > 0.0 ? tnorm / bnorm : 0.0;
  out[1] = bnorm > 0.0 ? gres / bnorm : 0.0;
  free(V); free(Z); free(H); free(cs); free(sn); free(g); free(yv); free(w);
  return status;
}

/* Right-preconditioned BiCGSTAB (van der Vorst, SIAM J. Sci. Stat. Comput.
 * 13, 1992), the Krylov method the paper pairs with Block Jacobi (Sec. 4.3).
 * The residual r is that of S x = b itself (right preconditioning, Sec. 2.2);
 * the shadow vector is r at the (re)start.  One pass is
 *   p  = r                         (first pass after a (re)start)
 *   p  = r + beta (p - omega v)    (later passes)
 *   ph = M^{-1} p,  v = S ph,  alpha = rho / (rt . v)
 *   x  = x + alpha ph,  s = r - alpha v     -- stop here if ||s|| <= tol
 *   sh = M^{-1} s,  t = S sh,  omega = (t . s) / (t . t)
 *   x  = x + omega sh,  r = s - omega t
 *   rho' = rt . r,  beta = (rho' / rho) (alpha / omega)
 * The count is the number of passes started.  A recurrence residual at the
 * tolerance (after either half) is confirmed with the true residual; if that
 * is still above it, the iteration restarts from r = b - S x.  Breakdown:
 * rt . v = 0, t . t = 0, omega = 0, rho' = 0, or a non-finite scalar. */
int or_bicgstab(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const or_precond* M,
                const double* b, double* x, double rtol, int64_t maxit, int64_t* iters, double* out) {
  size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double *r = (double*)malloc(sz), *rt = (double*)malloc(sz), *p = (double*)malloc(sz);
  double *ph = (double*)malloc(sz), *vv = (double*)malloc(sz), *sh = (double*)malloc(sz);
  double *t = (double*)malloc(sz);
  int status = OR_NOT_CONVERGED;
  int64_t it = 0;
  double bnorm = nrm2(n, b), tol = rtol * bnorm, rnorm = 0.0, tnorm = 0.0;
  or_spmv(n, rp, ci, v, x, t);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
  rnorm = tnorm = nrm2(n, r);
  if (bnorm == 0.0) { for (int64_t i = 0; i < n; ++i) x[i] = 0.0; rnorm = tnorm = 0.0; status = OR_OK; goto done; }
  if (rnorm <= tol) { status = OR_OK; goto done; }
  for (;;) {
    /* (re)start: shadow vector and rho from the current residual */
    memcpy(rt, r, sz);
    double rho = dot(n, rt, r), alpha = 0.0, omega = 0.0, beta = 0.0;
    int first = 1, reached = 0;
    while (it < maxit) {
      ++it;
      if (first) {
        memcpy(p, r, sz);
        first = 0;
      } else {
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * vv[i]);
      }
      precond_apply(M, p, ph);
      or_spmv(n, rp, ci, v, ph, vv);
      double rv = dot(n, rt, vv);
      if (rv == 0.0 || !isfinite(rv)) { status = OR_BREAKDOWN; break; }
      alpha = rho / rv;
      for (int64_t i = 0; i < n; ++i) { x[i] = x[i] + alpha * ph[i]; r[i] = r[i] - alpha * vv[i]; }
      rnorm = nrm2(n, r);
      if (rnorm <= tol) { reached = 1; break; }
      precond_apply(M, r, sh);
      or_spmv(n, rp, ci, v, sh, t);
      double tt = dot(n, t, t), ts = dot(n, t, r);
      if (!(tt > 0.0) || !isfinite(tt) || !isfinite(ts)) { status = OR_BREAKDOWN; break; }
      omega = ts / tt;
      for (int64_t i = 0; i < n; ++i) { x[i] = x[i] + omega * sh[i]; r[i] = r[i] - omega * t[i]; }
      rnorm = nrm2(n, r);
      if (rnorm <= tol) { reached = 1; break; }
      if (it >= maxit) break;
      double rho_new = dot(n, rt, r);
      if (rho_new == 0.0 || omega == 0.0 || !isfinite(rho_new) || !isfinite(omega)) { status = OR_BREAKDOWN; break; }
      beta = (rho_new / rho) * (alpha / omega);
      rho = rho_new;
    }
    if (!reached) break;
    or_spmv(n, rp, ci, v, x, t);
    for (int64_t i = 0; i < n; ++i) t[i] = b[i] - t[i];
    tnorm = nrm2(n, t);
    if (tnorm <= tol) { status = OR_OK; goto done; }
    if (it >= maxit) goto done;
    memcpy(r, t, sz);
    rnorm = tnorm;
  }
  or_spmv(n, rp, ci, v, x, t);
  for (int64_t i = 0; i < n; ++i) t[i] = b[i] - t[i];
  tnorm = nrm2(n, t);
done:
  *iters = it;
  out[0] = bnorm > 0.0 ? tnorm / bnorm : 0.0;
  out[1] = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  free(r); free(rt); free(p); free(ph); free(vv); free(sh); free(t);
  return status;
}

/* Restarted, right-preconditioned GCR(m) (Eisenstat, Elman and Schultz,
 * SIAM J. Numer. Anal. 20, 1983), the "IGCR(m)" the paper pairs with BBD
 * (Sec. 4.2, 4.3).  Step j of a cycle:
 *   p_j = M^{-1} r,  q_j = S p_j
 *   for i < j (modified Gram-Schmidt on the images):
 *       c = q_i . q_j,  q_j = q_j - c q_i,  p_j = p_j - c p_i
 *   d = ||q_j||,  q_j = q_j / d,  p_j = p_j / d
 *   a = q_j . r,  x = x + a p_j,  r = r - a q_j
 * so the q_i are orthonormal and S p_i = q_i; the iterate minimises
 * ||b - S x|| over the directions of the cycle.  The count is the number of
 * steps (products S p).  A cycle ends after m steps, on ||r|| <= rtol ||b||
 * (confirmed with the true residual; the next cycle starts from it) or when
 * q_j vanishes (breakdown). */
int or_gcr(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const or_precond* M,
           const double* b, double* x, double rtol, int64_t maxit, int64_t restart, int64_t* iters, double* out) {
  int64_t m = restart > 0 ? restart : 1;
  size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double* P = (double*)malloc(sz * (size_t)m);
  double* Q = (double*)malloc(sz * (size_t)m);
  double* r = (double*)malloc(sz);
  double* t = (double*)malloc(sz);
  int status = OR_NOT_CONVERGED;
  int64_t it = 0;
  double bnorm = nrm2(n, b), tol = rtol * bnorm, rnorm = 0.0, tnorm = 0.0;
  if (bnorm == 0.0) { for (int64_t i = 0; i < n; ++i) x[i] = 0.0; status = OR_OK; goto done; }
  for (;;) {
    or_spmv(n, rp, ci, v, x, t);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
    rnorm = tnorm = nrm2(n, r);
    if (tnorm <= tol) { status = OR_OK; break; }
    if (it >= maxit) break;
    int breakdown = 0;
    for (int64_t j = 0; j < m && it < maxit; ++j) {
      double* pj = P + j * n;
      double* qj = Q + j * n;
      precond_apply(M, r, pj);
      or_spmv(n, rp, ci, v, pj, qj);
      ++it;
      for (int64_t i = 0; i < j; ++i) {
        double c = dot(n, Q + i * n, qj);
        for (int64_t l = 0; l < n; ++l) { qj[l] = qj[l] - c * Q[i * n + l]; pj[l] = pj[l] - c * P[i * n + l]; }
      }
      double d = nrm2(n, qj);
      if (!(d > 0.0) || !isfinite(d)) { breakdown = 1; break; }
      for (int64_t l = 0; l < n; ++l) { qj[l] = qj[l] / d; pj[l] = pj[l] / d; }
      double a = dot(n, qj, r);
      for (int64_t l = 0; l < n; ++l) { x[l] = x[l] + a * pj[l]; r[l] = r[l] - a * qj[l]; }
      rnorm = nrm2(n, r);
      if (rnorm <= tol) break;
    }
    if (breakdown) { status = OR_BREAKDOWN; break; }
  }
  or_spmv(n, rp, ci, v, x, t);
  for (int64_t i = 0; i < n; ++i) t[i] = b[i] - t[i];
  tnorm = nrm2(n, t);
done:
  *iters = it;
  out[0] = bnorm > 0.0 ? tnorm / bnorm : 0.0;
  out[1] = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  free(P); free(Q); free(r); free(t);
  return status;
}

/* Entry points that build the preconditioner descriptor for Python callers. */
int or_pcg_bj(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const int64_t* prp,
              const int32_t* pci, const double* F, int64_t nblocks, const int64_t* block_ptr,
              const double* b, double* x, double rtol, int64_t maxit, int64_t* iters, double* out) {
  or_precond M = {1, n, prp, pci, NULL, F, nblocks, block_ptr, NULL, NULL};
  return or_pcg(n, rp, ci, v, &M, b, x, rtol, maxit, iters, out);
}

int or_gmres_bbd(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const int64_t* prp,
                 const int32_t* pci, const double* pv, const double* F, int64_t nblocks,
                 const int64_t* block_ptr, const double* lu, const int32_t* ipiv, const double* b,
                 double* x, double rtol, int64_t maxit, int64_t restart, int64_t* iters, double* out) {
  or_precond M = {3, n, prp, pci, pv, F, nblocks, block_ptr, lu, ipiv};
  return or_gmres(n, rp, ci, v, &M, b, x, rtol, maxit, restart, iters, out);
}

int or_gmres_pre(int kind, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                 const int64_t* prp, const int32_t* pci, const double* pv, const double* F,
                 int64_t nblocks, const int64_t* block_ptr, const double* lu, const int32_t* ipiv,
                 const double* b, double* x, double rtol, int64_t maxit, int64_t restart,
                 int64_t* iters, double* out) {
  or_precond M = {kind, n, prp, pci, pv, F, nblocks, block_ptr, lu, ipiv};
  return or_gmres(n, rp, ci, v, &M, b, x, rtol, maxit, restart, iters, out);
}

int or_bicgstab_pre(int kind, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                    const int64_t* prp, const int32_t* pci, const double* pv, const double* F,
                    int64_t nblocks, const int64_t* block_ptr, const double* b, double* x, double rtol,
                    int64_t maxit, int64_t* iters, double* out) {
  or_precond M = {kind, n, prp, pci, pv, F, nblocks, block_ptr, NULL, NULL};
  return or_bicgstab(n, rp, ci, v, &M, b, x, rtol, maxit, iters, out);
}

int or_gcr_pre(int kind, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
               const int64_t* prp, const int32_t* pci, const double* pv, const double* F,
               int64_t nblocks, const int64_t* block_ptr, const double* lu, const int32_t* ipiv,
               const double* b, double* x, double rtol, int64_t maxit, int64_t restart,
               int64_t* iters, double* out) {
  or_precond M = {kind, n, prp, pci, pv, F, nblocks, block_ptr, lu, ipiv};
  return or_gcr(n, rp, ci, v, &M, b, x, rtol, maxit, restart, iters, out);
}

void or_precond_apply(int kind, int64_t n, const int64_t* prp, const int32_t* pci, const double* pv,
                      const double* F, int64_t nblocks, const int64_t* block_ptr, const double* lu,
                      const int32_t* ipiv, const double* r, double* z) {
  or_precond M = {kind, n, prp, pci, pv, F, nblocks, block_ptr, lu, ipiv};
  precond_apply(&M, r, z);
}
