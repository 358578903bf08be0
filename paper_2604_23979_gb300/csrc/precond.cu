// precond.cu -- construction of the block preconditioner on the device.
//
//   filter      Eq. (filter), Algorithm 2: an off-diagonal p_ij is dropped iff
//               |p_ij| < tau|p_ii| and |p_ij| < tau|p_jj| (strict); diagonals stay.
//   correction  Eq. (diagcorr), Algorithm 3: p_ii + delta*sign(p_ii), sign(0)=+1.
//   scope       Block Jacobi keeps only entries inside the diagonal blocks
//               (Sec. 2.3); BBD keeps the whole matrix (Sec. 2.4).
//   levels      level sets of the in-block triangular solves (Sec. 2.3, fourth
//               step), one CTA per block (the blocks are independent units of
//               one launch).
//   IC(0)/ILU(0) per-block zero-fill factors (Sec. 2.3 third step; Sec. 3.1),
//               level-scheduled, one CTA per block, one warp per row.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace sdsl {

namespace {

inline unsigned grid_for(int64_t work, int per_block, int cap = 152 * 32) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

__global__ void k_diag_values(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const double* __restrict__ v, double* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = bsearch_i32(ci, rp[i], rp[i + 1], (int32_t)i);
    d[i] = p >= 0 ? v[p] : 0.0;
  }
}

__global__ void k_row_blocks(int64_t n, int64_t nblocks, const int64_t* __restrict__ bp, int32_t* __restrict__ rb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t b;
    if (i >= bp[nblocks]) {
      b = (int32_t)nblocks;
    } else {
      int64_t lo = 0, hi = nblocks;
      while (hi - lo > 1) { int64_t mid = (lo + hi) >> 1; if (bp[mid] <= i) lo = mid; else hi = mid; }
      b = (int32_t)lo;
    }
    rb[i] = b;
  }
}

// Warp per row.  kFill = false: prp[i] = kept count (missing diagonal counts
// as one).  kFill = true: write the kept entries in column order, the
// corrected diagonal, and pdiag[i].
template <bool kFill>
__global__ void k_filter(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const double* __restrict__ v, const double* __restrict__ d, const int32_t* __restrict__ rb,
                         int whole, double tau, double delta, int64_t* __restrict__ prp, int32_t* __restrict__ pci,
                         double* __restrict__ pv, int64_t* __restrict__ pdiag) {
  const int lane = lane_id();
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = wid; i < n; i += nw) {
    const int32_t bi = rb[i];
    const double ti = __dmul_rn(tau, fabs(d[i]));
    const int64_t s = rp[i], e = rp[i + 1];
    int kept = 0, below = 0;
    bool has_diag = false;
    for (int64_t base = s; base < e; base += 32) {
      const int64_t p = base + lane;
      bool keep = false, lo = false, dg = false;
      if (p < e) {
        const int32_t j = ci[p];
        if (whole || rb[j] == bi) {
          if (j == i) {
            keep = true; dg = true;
          } else {
            const double a = fabs(v[p]);
            keep = !(a < ti && a < __dmul_rn(tau, fabs(d[j])));
            lo = keep && j < i;
          }
        }
      }
      kept += __popc(__ballot_sync(0xffffffffu, keep));
      below += __popc(__ballot_sync(0xffffffffu, lo));
      has_diag |= __ballot_sync(0xffffffffu, dg) != 0;
    }
    if (!kFill) {
      if (lane == 0) prp[i] = kept + (has_diag ? 0 : 1);
      continue;
    }
    const int64_t out0 = prp[i];
    if (!has_diag && lane == 0) {
      pci[out0 + below] = (int32_t)i;
      pv[out0 + below] = __dadd_rn(0.0, delta);
      pdiag[i] = out0 + below;
    }
    int64_t run = 0;
    for (int64_t base = s; base < e; base += 32) {
      const int64_t p = base + lane;
      bool keep = false;
      int32_t j = 0;
      double val = 0.0;
      if (p < e) {
        j = ci[p];
        val = v[p];
        if (whole || rb[j] == bi) {
          if (j == i) {
            keep = true;
          } else {
            const double a = fabs(val);
            keep = !(a < ti && a < __dmul_rn(tau, fabs(d[j])));
          }
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        int64_t at = out0 + run + __popc(mask & ((1u << lane) - 1u));
        if (!has_diag && j > i) at += 1;
        pci[at] = j;
        if (j == i) {
          const double sg = val < 0.0 ? -1.0 : 1.0;
          pv[at] = __dadd_rn(val, __dmul_rn(delta, sg));
          pdiag[i] = at;
        } else {
          pv[at] = val;
        }
      }
      run += __popc(mask);
    }
  }
}

__global__ void k_mirror_map(int64_t n, const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                             const int64_t* __restrict__ pdiag, int64_t* __restrict__ mir, int* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t t = pdiag[i] + 1; t < prp[i + 1]; ++t) {
      const int32_t j = pci[t];
      const int64_t q = bsearch_i32(pci, prp[j], pdiag[j], (int32_t)i);
      mir[t] = q;
      if (q < 0) atomicExch(bad, 1);
    }
  }
}

// Level sets by layered topological order (Kahn), one CTA per block.
// dir = 0: row i depends on in-block j < i of its row (lower solve); the rows
// released by j are the in-block entries right of j's diagonal (the pattern
// is symmetric).  dir = 1: mirror image (upper solve, last row first).
__global__ void k_levels(int dir, const int64_t* __restrict__ bp, const int64_t* __restrict__ prp,
                         const int32_t* __restrict__ pci, const int64_t* __restrict__ pdiag, int32_t* __restrict__ cnt,
                         int32_t* __restrict__ lev, int32_t* __restrict__ fa, int32_t* __restrict__ fb,
                         int32_t* __restrict__ nlev) {
  const int64_t s = bp[blockIdx.x], e = bp[blockIdx.x + 1];
  __shared__ int32_t nfront, nnext;
  if (threadIdx.x == 0) { nfront = 0; nnext = 0; }
  __syncthreads();
  for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x) {
    int32_t c = 0;
    if (dir == 0) {
      for (int64_t t = prp[i]; t < pdiag[i]; ++t) c += pci[t] >= s;
    } else {
      for (int64_t t = pdiag[i] + 1; t < prp[i + 1]; ++t) c += pci[t] < e;
    }
    cnt[i] = c;
    lev[i] = -1;
    if (c == 0) {
      lev[i] = 0;
      fa[s + atomicAdd(&nfront, 1)] = (int32_t)i;
    }
  }
  __syncthreads();
  int32_t level = 0;
  int32_t* cur = fa;
  int32_t* nxt = fb;
  while (nfront > 0) {
    const int32_t nf = nfront;
    for (int32_t k = threadIdx.x; k < nf; k += blockDim.x) {
      const int64_t j = cur[s + k];
      const int64_t t0 = dir == 0 ? pdiag[j] + 1 : prp[j];
      const int64_t t1 = dir == 0 ? prp[j + 1] : pdiag[j];
      for (int64_t t = t0; t < t1; ++t) {
        const int32_t i = pci[t];
        if (i < s || i >= e) continue;
        if (atomicSub(&cnt[i], 1) == 1) {
          lev[i] = level + 1;
          nxt[s + atomicAdd(&nnext, 1)] = i;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) { nfront = nnext; nnext = 0; }
    ++level;
    int32_t* tmp = cur; cur = nxt; nxt = tmp;
    __syncthreads();
  }
  if (threadIdx.x == 0) nlev[blockIdx.x] = (e > s) ? level : 0;
}

// Level lists of block b: counting sort of its rows by level, rows ascending
// inside each level.  level_ptr[lev_off[b] + l] = start of level l (absolute
// offset into level_rows); the caller sets level_ptr[total] = bp[nblocks].
__global__ void k_level_lists(const int64_t* __restrict__ bp, const int32_t* __restrict__ lev,
                              const int32_t* __restrict__ lev_off, int32_t* __restrict__ hist,
                              int32_t* __restrict__ level_ptr, int32_t* __restrict__ level_rows) {
  const int64_t s = bp[blockIdx.x], e = bp[blockIdx.x + 1];
  const int32_t off = lev_off[blockIdx.x];
  const int32_t nl = lev_off[blockIdx.x + 1] - off;
  for (int64_t l = threadIdx.x; l < nl; l += blockDim.x) hist[s + l] = 0;
  __syncthreads();
  for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x)
    if (lev[i] >= 0 && lev[i] < nl) atomicAdd(&hist[s + lev[i]], 1);
  __syncthreads();
  if (threadIdx.x < 32) {  // warp 0: exclusive scan of the histogram, then stable placement
    const int lane = threadIdx.x;
    int32_t carry = 0;
    for (int64_t base = 0; base < nl; base += 32) {
      const int64_t l = base + lane;
      int32_t x = l < nl ? hist[s + l] : 0, inc = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (l < nl) {
        hist[s + l] = carry + inc - x;  // now the cursor of level l (relative to s)
        level_ptr[off + l] = (int32_t)s + carry + inc - x;
      }
      carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    __syncwarp();
    for (int64_t base = s; base < e; base += 32) {
      const int64_t i = base + lane;
      const bool act = i < e;
      const unsigned amask = __ballot_sync(0xffffffffu, act);
      if (act) {
        const int32_t L = lev[i];
        const unsigned peers = __match_any_sync(amask, L);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const int32_t cur = hist[s + L];
        level_rows[s + cur + rank] = (int32_t)i;
        __syncwarp(amask);
        if (rank == 0) hist[s + L] = cur + __popc(peers);
      }
      __syncwarp();
    }
  }
}

// IC(0), row oriented: for each k < i of row i (ascending),
//   l_ik = (p_ik - sum_{j<k} l_ij l_kj) / l_kk,  l_ii = sqrt(p~_ii - sum l_ij^2),
// p~_ii = p_ii + alpha p_ii (shift of the retry rule).  Rows of one level are
// independent; a warp takes one row and keeps its columns and values in
// shared memory while lanes split the inner products over row k.
// Grid: nblocks x nshift CTAs; CTA (b, t) factors block b with shift
// alpha[t] into F + t * nnz (all shifts of the retry ladder run at once).
constexpr int kIcWarps = 32;
constexpr int kIcCap = 192;  // row entries staged in shared memory per warp
__global__ void __launch_bounds__(kIcWarps * 32) k_ic0(const int64_t* __restrict__ bp, const int64_t* __restrict__ prp,
                      const int32_t* __restrict__ pci, const double* __restrict__ pv,
                      const int64_t* __restrict__ pdiag, const int32_t* __restrict__ lev_off,
                      const int32_t* __restrict__ level_ptr, const int32_t* __restrict__ level_rows,
                      const double* __restrict__ alpha, int nshift, int64_t nnz, int64_t n,
                      double* __restrict__ Fall, double* __restrict__ dinv_all, int32_t* __restrict__ status,
                      const int32_t* __restrict__ order) {
  // blocks in the given order (largest first: the longest factorizations
  // start in the first wave of CTAs)
  const int b = order ? order[blockIdx.x / nshift] : (int)(blockIdx.x / nshift), sh = blockIdx.x % nshift;
  double* __restrict__ F = Fall + (int64_t)sh * nnz;
  double* __restrict__ dinv = dinv_all + (int64_t)sh * n;
  const int64_t s = bp[b];
  const double al = alpha[sh];
  __shared__ int failed;
  __shared__ int32_t scol[kIcWarps][kIcCap];
  __shared__ double sval[kIcWarps][kIcCap];
  if (threadIdx.x == 0) failed = 0;
  __syncthreads();
  const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int32_t L = lev_off[b]; L < lev_off[b + 1]; ++L) {
    const int32_t r0 = level_ptr[L], r1 = level_ptr[L + 1];
    for (int32_t idx = r0 + w; idx < r1; idx += nw) {
      const int64_t i = level_rows[idx];
      const int64_t lo = prp[i], dg = pdiag[i];
      int64_t t0 = lo;
      while (t0 < dg && pci[t0] < s) ++t0;  // first in-block entry
      const int64_t len = dg - t0;
      const bool staged = len <= kIcCap;
      int32_t* cols = scol[w];
      double* vals = sval[w];
      if (staged)
        for (int64_t q = lane; q < len; q += 32) cols[q] = pci[t0 + q];
      __syncwarp();
      // Software pipeline over the row's entries t: row k_{t+1}'s pattern,
      // its first 32 entries and its diagonal are loaded while entry t is
      // computed (row k_{t+1} belongs to an earlier level, so they are final);
      // every lane still sums its entries q = prp[k] + lane, +32, ... in order.
      int64_t kd_c = 0, q0_c = 0;
      int32_t j_c = -1;
      double f_c = 0.0, d_c = 1.0;
      auto fetch = [&](int64_t t, int64_t& q0, int64_t& kd, int32_t& j, double& f, double& d) {
        const int64_t k = pci[t0 + t];
        q0 = prp[k];
        kd = pdiag[k];
        const int64_t q = q0 + lane;
        j = q < kd ? pci[q] : -1;
        f = q < kd ? F[q] : 0.0;
        d = F[kd];
      };
      if (len > 0) fetch(0, q0_c, kd_c, j_c, f_c, d_c);
      for (int64_t t = 0; t < len; ++t) {
        int64_t kd_n = 0, q0_n = 0;
        int32_t j_n = -1;
        double f_n = 0.0, d_n = 1.0;
        if (t + 1 < len) fetch(t + 1, q0_n, kd_n, j_n, f_n, d_n);
        double acc = 0.0;
        if (j_c >= s) {
          const int64_t pos = staged ? bsearch_i32(cols, 0, t, j_c) : bsearch_i32(pci + t0, 0, t, j_c);
          if (pos >= 0) acc = __fma_rn(staged ? vals[pos] : F[t0 + pos], f_c, acc);
        }
        for (int64_t q = q0_c + lane + 32; q < kd_c; q += 32) {
          const int32_t j = pci[q];
          if (j < s) continue;
          const int64_t pos = staged ? bsearch_i32(cols, 0, t, j) : bsearch_i32(pci + t0, 0, t, j);
          if (pos >= 0) acc = __fma_rn(staged ? vals[pos] : F[t0 + pos], F[q], acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) {
          const double l = (pv[t0 + t] - acc) / d_c;
          if (staged) vals[t] = l; else F[t0 + t] = l;
        }
        __syncwarp();
        kd_c = kd_n;
        q0_c = q0_n;
        j_c = j_n;
        f_c = f_n;
        d_c = d_n;
      }
      double sq = 0.0;
      for (int64_t q = lane; q < len; q += 32) {
        const double l = staged ? vals[q] : F[t0 + q];
        sq = __fma_rn(l, l, sq);
        if (staged) F[t0 + q] = l;
      }
      sq = warp_sum(sq);
      if (lane == 0) {
        const double pd = al == 0.0 ? pv[dg] : __dadd_rn(pv[dg], __dmul_rn(al, pv[dg]));
        const double dd = pd - sq;
        if (!(dd > 0.0) || !isfinite(dd)) {
          failed = 1;
          F[dg] = 1.0;
          dinv[i] = 1.0;
        } else {
          const double l = sqrt(dd);
          F[dg] = l;
          dinv[i] = 1.0 / l;
        }
      }
      __syncwarp();
    }
    __syncthreads();
    if (failed) break;
  }
  if (threadIdx.x == 0) status[b * nshift + sh] = failed;
}

// Copy the factor of the chosen shift of every block into F / dinv.
__global__ void k_pick_shift(const int64_t* __restrict__ bp, const int64_t* __restrict__ prp,
                             const int32_t* __restrict__ choice, int64_t nnz, int64_t n,
                             const double* __restrict__ Fall, const double* __restrict__ dinv_all,
                             double* __restrict__ F, double* __restrict__ dinv, const int32_t* __restrict__ rb,
                             int64_t nrows) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = choice[rb[i]];
    for (int64_t t = prp[i]; t < prp[i + 1]; ++t) F[t] = Fall[(int64_t)c * nnz + t];
    dinv[i] = dinv_all[(int64_t)c * n + i];
  }
}

// ILU(0), IKJ order restricted to the in-block pattern: for each k < i of row
// i (ascending), l_ik = w_ik / u_kk, then w_ij -= l_ik u_kj for the j > k of
// row i present in row k.  Unit L stored at j < i, U at j >= i.
__global__ void k_ilu0(const int64_t* __restrict__ bp, const int64_t* __restrict__ prp,
                       const int32_t* __restrict__ pci, const double* __restrict__ pv,
                       const int64_t* __restrict__ pdiag, const int32_t* __restrict__ lev_off,
                       const int32_t* __restrict__ level_ptr, const int32_t* __restrict__ level_rows,
                       const double* __restrict__ alpha, const int32_t* __restrict__ active, double* __restrict__ F,
                       double* __restrict__ dinv, int32_t* __restrict__ status) {
  const int b = blockIdx.x;
  if (!active[b]) return;
  const int64_t s = bp[b], e = bp[b + 1];
  const double al = alpha[b];
  __shared__ int failed;
  if (threadIdx.x == 0) failed = 0;
  __syncthreads();
  const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int32_t L = lev_off[b]; L < lev_off[b + 1]; ++L) {
    const int32_t r0 = level_ptr[L], r1 = level_ptr[L + 1];
    for (int32_t idx = r0 + w; idx < r1; idx += nw) {
      const int64_t i = level_rows[idx];
      const int64_t lo = prp[i], hi = prp[i + 1], dg = pdiag[i];
      for (int64_t t = lo + lane; t < hi; t += 32) {
        const int32_t j = pci[t];
        if (j >= s && j < e) F[t] = (t == dg) ? (al == 0.0 ? pv[t] : __dadd_rn(pv[t], __dmul_rn(al, pv[t]))) : pv[t];
      }
      __syncwarp();
      for (int64_t t = lo; t < dg; ++t) {
        const int64_t k = pci[t];
        if (k < s) continue;
        const double lik = F[t] / F[pdiag[k]];
        __syncwarp();
        if (lane == 0) F[t] = lik;
        const int64_t kd = pdiag[k], ke = prp[k + 1];
        for (int64_t q = t + 1 + lane; q < hi; q += 32) {
          const int32_t j = pci[q];
          if (j >= e) continue;
          const int64_t kq = bsearch_i32(pci, kd + 1, ke, j);
          if (kq >= 0) F[q] = __dsub_rn(F[q], __dmul_rn(lik, F[kq]));
        }
        __syncwarp();
      }
      if (lane == 0) {
        const double u = F[dg];
        if (u == 0.0 || !isfinite(u)) { failed = 1; dinv[i] = 1.0; } else { dinv[i] = 1.0 / u; }
      }
      __syncwarp();
    }
    __syncthreads();
    if (failed) break;
  }
  if (threadIdx.x == 0) status[b] = failed;
}

// One thread per position q of the level lists: row i = lev_rows[q] of block
// b = row_block[i]; its in-block strict entries in the solve direction.
__global__ void k_pack_count(int dir, int64_t npos, const int32_t* __restrict__ rb, const int64_t* __restrict__ bp,
                             const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                             const int64_t* __restrict__ pdiag, const int32_t* __restrict__ lev_rows,
                             int64_t* __restrict__ off) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npos; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = lev_rows[q];
    if (i < 0) { off[q] = 0; continue; }  // padding position
    const int32_t b = rb[i];
    const int64_t s = bp[b], e = bp[b + 1];
    int64_t c = 0;
    if (dir == 0) {
      for (int64_t t = prp[i]; t < pdiag[i]; ++t) c += pci[t] >= s;
    } else {
      for (int64_t t = pdiag[i] + 1; t < prp[i + 1]; ++t) c += pci[t] < e;
    }
    off[q] = c;
  }
}

template <typename TS>
__global__ void k_pack_fill(int dir, int64_t npos, const int32_t* __restrict__ rb, const int64_t* __restrict__ bp,
                            const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                            const int64_t* __restrict__ pdiag, const int32_t* __restrict__ lev_rows,
                            const double* __restrict__ F, const double* __restrict__ dinv,
                            const int64_t* __restrict__ off, int32_t* __restrict__ col, TS* __restrict__ val,
                            TS* __restrict__ pdinv, int32_t* __restrict__ prow) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npos; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = lev_rows[q];
    if (i < 0) {  // padding position: no entries, no row
      pdinv[q] = (TS)1;
      prow[q] = -1;
      continue;
    }
    const int32_t b = rb[i];
    const int64_t s = bp[b], e = bp[b + 1];
    int64_t at = off[q];
    const int64_t t0 = dir == 0 ? prp[i] : pdiag[i] + 1;
    const int64_t t1 = dir == 0 ? pdiag[i] : prp[i + 1];
    for (int64_t t = t0; t < t1; ++t) {
      const int32_t j = pci[t];
      if (j < s || j >= e) continue;
      col[at] = (int32_t)(j - s);
      val[at] = (TS)F[t];
      ++at;
    }
    pdinv[q] = (TS)dinv[i];
    prow[q] = (int32_t)(i - s);
  }
}

// Byte sizes of the staged tile streams are multiples of 16.
__host__ __device__ inline int64_t r16(int64_t x) { return (x + 15) & ~(int64_t)15; }

// Strict in-block entries of row i (dir 0: lower, 1: upper) of block [s, e).

__device__ __forceinline__ int strict_count(int dir, int64_t i, int64_t s, int64_t e, const int64_t* prp,
                                            const int32_t* pci, const int64_t* pdiag) {
  int c = 0;
  if (dir == 0) {
    for (int64_t t = prp[i]; t < pdiag[i]; ++t) c += pci[t] >= s;
  } else {
    for (int64_t t = pdiag[i] + 1; t < prp[i + 1]; ++t) c += pci[t] < e;
  }
  return c;
}

// Variable-width tiles.  A tile holds rows of one level L (within its
// block); row r of the tile gets V_r lanes (a power of two, a planned number
// of entries per lane), groups packed at V-aligned lane offsets.  A row's
// strict in-block entries are split by the level of their column: "near"
// (levels L - gap + 1 .. L - 1: the values the row waits for last) and "far"
// (level <= L - gap, usually final long before).  The row's near entries come first, all read by
// the row's first lane (its leader); then its far entries, dealt to the V
// lanes round-robin (lane k reads far entries k, k + V, ...).  Each group is
// in ascending column order.  Layout (16-byte aligned parts):
//   int32 nr, ne, L, (tiles of level L-1) | (tiles of level L-gap) << 16
//   lane record x 32 (8 bytes each): uint16 row (block-local; 0xFFFF = idle),
//     uint16 first (index of the lane's first far entry in the tile), uint8
//     far count of the lane, uint8 log2 V, uint8 r | leader << 7 (r = row
//     within the tile), uint8 near count (leader; its near entries are the
//     ones just before `first`)
//   TS dinv[nr] | uint16 col[ne] (block-local) | TS val[ne]
// A lane reads its whole role with one 8-byte load.  The plan (rows of every
// tile in packing order and their V) is built on the host; one tile per
// thread.  *bad is set if a row has more than 255 near entries.
// Stored factor value from the FP64 factor: FP64, FP32, or BF16 through FP32
// (so the BF16 values equal those of the rounded FP32 copy).
template <typename TS>
__device__ __forceinline__ TS to_stored(double v) { return (TS)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_stored<__nv_bfloat16>(double v) {
  return __float2bfloat16_rn((float)v);
}

template <typename TS>
__global__ void k_vt_fill(int dir, int64_t ntiles, const int32_t* __restrict__ tile_rows_ptr,
                          const int32_t* __restrict__ plan_rows, const int8_t* __restrict__ plan_logv,
                          const int32_t* __restrict__ rb, const int64_t* __restrict__ bp,
                          const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                          const int64_t* __restrict__ pdiag, const double* __restrict__ F,
                          const double* __restrict__ dinv, const int32_t* __restrict__ lev,
                          const int64_t* __restrict__ toff, const int32_t* __restrict__ tile_meta,
                          unsigned char* __restrict__ stream, int* __restrict__ bad, int gap) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
    unsigned char* base = stream + toff[t];
    const int r0 = tile_rows_ptr[t], nr = tile_rows_ptr[t + 1] - r0;
    int32_t* hdr = reinterpret_cast<int32_t*>(base);
    uint16_t* rec = reinterpret_cast<uint16_t*>(base + 16);
    TS* dv = reinterpret_cast<TS*>(base + 16 + 256);
    for (int l = 0; l < 32; ++l) {
      rec[4 * l + 0] = 0xFFFFu;
      rec[4 * l + 1] = 0;
      rec[4 * l + 2] = 0;
      rec[4 * l + 3] = 0;
    }
    int lane = 0, ne = 0;
    for (int r = 0; r < nr; ++r) {
      const int64_t i = plan_rows[r0 + r];
      const int lv = plan_logv[r0 + r], V = 1 << lv;
      const int32_t b = rb[i];
      const int64_t s = bp[b], e = bp[b + 1];
      const int len = strict_count(dir, i, s, e, prp, pci, pdiag);
      const int64_t t0 = dir == 0 ? prp[i] : pdiag[i] + 1;
      const int64_t t1 = dir == 0 ? pdiag[i] : prp[i + 1];
      int nfar = 0;
      for (int64_t q = t0; q < t1; ++q) {
        const int32_t j = pci[q];
        if (j >= s && j < e && lev[j] <= lev[i] - gap) ++nfar;
      }
      const int nnear = len - nfar;
      if (nnear > 255) *bad = 1;
      dv[r] = to_stored<TS>(dinv[i]);
      for (int k = 0; k < V; ++k) {
        const int cfar = k < nfar ? (nfar - k + V - 1) / V : 0;
        rec[4 * (lane + k) + 0] = (uint16_t)(i - s);
        rec[4 * (lane + k) + 1] = (uint16_t)(ne + nnear + k);
        rec[4 * (lane + k) + 2] = (uint16_t)(cfar | (lv << 8));
        rec[4 * (lane + k) + 3] = (uint16_t)(r | (k == 0 ? 0x80 | ((nnear & 0xFF) << 8) : 0));
      }
      lane += V;
      ne += len;
    }
    hdr[0] = nr;
    hdr[1] = ne;
    hdr[2] = tile_meta ? tile_meta[3 * t] : 0;  // level of the tile within its block
    hdr[3] = tile_meta ? (tile_meta[3 * t + 1] | (tile_meta[3 * t + 2] << 16)) : 0;
    uint16_t* col = reinterpret_cast<uint16_t*>(base + 16 + 256 + r16((int64_t)nr * sizeof(TS)));
    TS* val = reinterpret_cast<TS*>(reinterpret_cast<unsigned char*>(col) + r16(2 * (int64_t)ne));
    int at = 0;
    for (int r = 0; r < nr; ++r) {
      const int64_t i = plan_rows[r0 + r];
      const int32_t b = rb[i];
      const int64_t s = bp[b], e = bp[b + 1];
      const int64_t t0 = dir == 0 ? prp[i] : pdiag[i] + 1;
      const int64_t t1 = dir == 0 ? pdiag[i] : prp[i + 1];
      for (int pass = 0; pass < 2; ++pass) {  // near entries, then far ones
        for (int64_t q = t0; q < t1; ++q) {
          const int32_t j = pci[q];
          if (j < s || j >= e) continue;
          if ((lev[j] <= lev[i] - gap) != (pass == 1)) continue;
          col[at] = (uint16_t)(j - s);
          val[at] = to_stored<TS>(F[q]);
          ++at;
        }
      }
    }
  }
}

__global__ void k_ic0_finish(int64_t n, const int64_t* __restrict__ prp, const int64_t* __restrict__ pdiag,
                             const int64_t* __restrict__ mir, double* __restrict__ F) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t t = pdiag[i] + 1; t < prp[i + 1]; ++t) F[t] = F[mir[t]];
}

// FP32 values rounded to BF16 precision in place (the stored BF16 factor,
// widened, for exports and checks).
__global__ void k_round_bf16(int64_t n, float* __restrict__ a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = __bfloat162float(__float2bfloat16_rn(a[i]));
}

__global__ void k_to_float(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

}  // namespace

cudaError_t diag_values(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, double* d, cudaStream_t st) {
  k_diag_values<<<grid_for(n, 256), 256, 0, st>>>(n, rp, ci, v, d); count_launch();
  return cudaGetLastError();
}

cudaError_t row_blocks(int64_t n, int64_t nblocks, const int64_t* bp, int32_t* row_block, cudaStream_t st) {
  k_row_blocks<<<grid_for(n, 256), 256, 0, st>>>(n, nblocks, bp, row_block); count_launch();
  return cudaGetLastError();
}

cudaError_t filter_count(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* d,
                         const int32_t* row_block, const int64_t* bp, int whole, double tau, int64_t* prp,
                         cudaStream_t st) {
  (void)bp;
  k_filter<false><<<grid_for(n, 8), 256, 0, st>>>(n, rp, ci, v, d, row_block, whole, tau, 0.0, prp, nullptr, nullptr,
                                                  nullptr); count_launch();
  return cudaGetLastError();
}

cudaError_t filter_fill(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* d,
                        const int32_t* row_block, const int64_t* bp, int whole, double tau, double delta,
                        const int64_t* prp, int32_t* pci, double* pv, int64_t* pdiag, cudaStream_t st) {
  (void)bp;
  k_filter<true><<<grid_for(n, 8), 256, 0, st>>>(n, rp, ci, v, d, row_block, whole, tau, delta,
                                                 const_cast<int64_t*>(prp), pci, pv, pdiag); count_launch();
  return cudaGetLastError();
}

cudaError_t mirror_map(int64_t n, const int64_t* prp, const int32_t* pci, const int64_t* pdiag, int64_t* mir,
                       int* bad, cudaStream_t st) {
  k_mirror_map<<<grid_for(n, 256), 256, 0, st>>>(n, prp, pci, pdiag, mir, bad); count_launch();
  return cudaGetLastError();
}

cudaError_t levels(int dir, int64_t nblocks, const int64_t* bp, const int64_t* prp, const int32_t* pci,
                   const int64_t* pdiag, int32_t* cnt, int32_t* lev, int32_t* fa, int32_t* fb, int32_t* nlev,
                   cudaStream_t st) {
  if (nblocks == 0) return cudaSuccess;
  k_levels<<<(unsigned)nblocks, 512, 0, st>>>(dir, bp, prp, pci, pdiag, cnt, lev, fa, fb, nlev); count_launch();
  return cudaGetLastError();
}

cudaError_t level_lists(int64_t nblocks, const int64_t* bp, const int32_t* lev, const int32_t* lev_off,
                        int32_t* hist, int32_t* level_ptr, int32_t* level_rows, cudaStream_t st) {
  if (nblocks == 0) return cudaSuccess;
  k_level_lists<<<(unsigned)nblocks, 256, 0, st>>>(bp, lev, lev_off, hist, level_ptr, level_rows); count_launch();
  return cudaGetLastError();
}

cudaError_t ic0_factor_all(int64_t nblocks, const int64_t* bp, const int64_t* prp, const int32_t* pci,
                           const double* pv, const int64_t* pdiag, const int32_t* lev_off, const int32_t* level_ptr,
                           const int32_t* level_rows, const double* alpha, int nshift, int64_t nnz, int64_t n,
                           double* Fall, double* dinv_all, int32_t* status, const int32_t* order,
                           cudaStream_t st) {
  if (nblocks == 0) return cudaSuccess;
  k_ic0<<<(unsigned)(nblocks * nshift), kIcWarps * 32, 0, st>>>(bp, prp, pci, pv, pdiag, lev_off, level_ptr,
                                                               level_rows, alpha, nshift, nnz, n, Fall, dinv_all,
                                                               status, order); count_launch();
  return cudaGetLastError();
}

cudaError_t pick_shift(const int64_t* bp, const int64_t* prp, const int32_t* choice, int64_t nnz, int64_t n,
                       const double* Fall, const double* dinv_all, double* F, double* dinv, const int32_t* rb,
                       int64_t nrows, cudaStream_t st) {
  k_pick_shift<<<grid_for(nrows, 256), 256, 0, st>>>(bp, prp, choice, nnz, n, Fall, dinv_all, F, dinv, rb, nrows); count_launch();
  return cudaGetLastError();
}

cudaError_t ilu0_factor(int64_t nblocks, const int64_t* bp, const int64_t* prp, const int32_t* pci, const double* pv,
                        const int64_t* pdiag, const int32_t* lev_off, const int32_t* level_ptr,
                        const int32_t* level_rows, const double* alpha, const int32_t* active, double* F,
                        double* dinv, int32_t* status, cudaStream_t st) {
  if (nblocks == 0) return cudaSuccess;
  k_ilu0<<<(unsigned)nblocks, 1024, 0, st>>>(bp, prp, pci, pv, pdiag, lev_off, level_ptr, level_rows, alpha, active,
                                             F, dinv, status); count_launch();
  return cudaGetLastError();
}

cudaError_t ic0_finish(int64_t n, int64_t nnz, const int64_t* prp, const int64_t* pdiag, const int64_t* mir,
                       double* F, const double* dinv, float* Ff, float* dinvf, cudaStream_t st) {
  k_ic0_finish<<<grid_for(n, 256), 256, 0, st>>>(n, prp, pdiag, mir, F); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  if (Ff) {
    k_to_float<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, F, Ff); count_launch();
    SDSL_CUDA_TRY(cudaGetLastError());
    k_to_float<<<grid_for(n, 256), 256, 0, st>>>(n, dinv, dinvf); count_launch();
    SDSL_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

cudaError_t pack_count(int dir, int64_t npos, const int32_t* row_block, const int64_t* bp, const int64_t* prp,
                       const int32_t* pci, const int64_t* pdiag, const int32_t* lev_rows, int64_t* off,
                       cudaStream_t st) {
  k_pack_count<<<grid_for(npos, 256), 256, 0, st>>>(dir, npos, row_block, bp, prp, pci, pdiag, lev_rows, off); count_launch();
  return cudaGetLastError();
}

cudaError_t pack_fill(int dir, int64_t npos, const int32_t* row_block, const int64_t* bp, const int64_t* prp,
                      const int32_t* pci, const int64_t* pdiag, const int32_t* lev_rows, const double* F,
                      const double* dinv, int prec, const int64_t* off, int32_t* col, void* val, void* pdinv,
                      int32_t* prow, cudaStream_t st) {
  if (prec == 32) {
    k_pack_fill<float><<<grid_for(npos, 256), 256, 0, st>>>(dir, npos, row_block, bp, prp, pci, pdiag, lev_rows, F,
                                                            dinv, off, col, static_cast<float*>(val),
                                                            static_cast<float*>(pdinv), prow); count_launch();
  } else {
    k_pack_fill<double><<<grid_for(npos, 256), 256, 0, st>>>(dir, npos, row_block, bp, prp, pci, pdiag, lev_rows,
                                                             F, dinv, off, col, static_cast<double*>(val),
                                                             static_cast<double*>(pdinv), prow); count_launch();
  }
  return cudaGetLastError();
}

cudaError_t vt_fill(int dir, int64_t ntiles, const int32_t* tile_rows_ptr, const int32_t* plan_rows,
                    const int8_t* plan_logv, const int32_t* row_block, const int64_t* bp, const int64_t* prp,
                    const int32_t* pci, const int64_t* pdiag, const double* F, const double* dinv, const int32_t* lev,
                    int prec, const int64_t* toff, const int32_t* tile_meta, unsigned char* stream, int* bad,
                    int gap, cudaStream_t st) {
  if (prec == 16) {
    k_vt_fill<__nv_bfloat16><<<grid_for(ntiles, 128), 128, 0, st>>>(dir, ntiles, tile_rows_ptr, plan_rows,
                                                                    plan_logv, row_block, bp, prp, pci, pdiag, F,
                                                                    dinv, lev, toff, tile_meta, stream, bad, gap);
    count_launch();
  } else if (prec == 32) {
    k_vt_fill<float><<<grid_for(ntiles, 128), 128, 0, st>>>(dir, ntiles, tile_rows_ptr, plan_rows, plan_logv,
                                                            row_block, bp, prp, pci, pdiag, F, dinv, lev, toff,
                                                            tile_meta, stream, bad, gap); count_launch();
  } else {
    k_vt_fill<double><<<grid_for(ntiles, 128), 128, 0, st>>>(dir, ntiles, tile_rows_ptr, plan_rows, plan_logv,
                                                             row_block, bp, prp, pci, pdiag, F, dinv, lev, toff,
                                                             tile_meta, stream, bad, gap); count_launch();
  }
  return cudaGetLastError();
}

cudaError_t round_bf16(int64_t n, float* a, cudaStream_t st) {
  k_round_bf16<<<grid_for(n, 256), 256, 0, st>>>(n, a); count_launch();
  return cudaGetLastError();
}

cudaError_t to_float(int64_t n, const double* a, float* b, cudaStream_t st) {
  k_to_float<<<grid_for(n, 256), 256, 0, st>>>(n, a, b); count_launch();
  return cudaGetLastError();
}

}  // namespace sdsl
