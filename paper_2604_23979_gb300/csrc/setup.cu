// setup.cu -- formation of the system matrix on the device.
//
// Normal equations (Eq. schur): S = A diag(theta) A^T + rho I.  The pattern
// (symbolic product) is built once per A, the values on every new theta
// (preconditioner reuse, Sec. 3.4).  Values follow one fixed rounding order,
// identical to the CPU oracle's, so that the filtered pattern is bit-exact:
// for (i, j) with h = max(i,j), l = min(i,j), acc = fma(fl(a_hk*theta_k), a_lk,
// acc) over shared columns k ascending, from +0; then S_ii = acc + rho.
//
// Augmented form (Eq. augmented): K = [[-diag(1/theta), A^T], [A, rho I]] in
// bordered block-diagonal order (Sec. 2.4).
#include "common.cuh"
#include "kernels.cuh"

namespace sdsl {

namespace {

constexpr int kSymCap = 1024;      // candidates per row handled by one warp
constexpr int kLongCap = 16384;    // candidates per row handled by one CTA
constexpr int kSetupWarps = 8;

__global__ void k_transpose_count(int64_t m, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                  unsigned long long* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) atomicAdd(&cnt[ci[p]], 1ull);
}

__global__ void k_transpose_fill(int64_t m, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const double* __restrict__ v, unsigned long long* __restrict__ cursor,
                                 int32_t* __restrict__ tci, double* __restrict__ tv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int64_t q = (int64_t)atomicAdd(&cursor[ci[p]], 1ull);
      tci[q] = (int32_t)i;
      if (tv) tv[q] = v[p];
    }
}

// Sort each row segment of (col, val) by column (insertion sort; short rows).
__global__ void k_sort_segments(int64_t n, const int64_t* __restrict__ rp, int32_t* __restrict__ ci,
                                double* __restrict__ v) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rp[r], e = rp[r + 1];
    for (int64_t a = s + 1; a < e; ++a) {
      int32_t c = ci[a];
      double x = v ? v[a] : 0.0;
      int64_t b = a - 1;
      while (b >= s && ci[b] > c) {
        ci[b + 1] = ci[b];
        if (v) v[b + 1] = v[b];
        --b;
      }
      ci[b + 1] = c;
      if (v) v[b + 1] = x;
    }
  }
}

// Bitonic sort of buf[0, P) (P a power of two) by `nthr` cooperating threads.
template <bool kBlock>
__device__ void bitonic_sort(int32_t* buf, int P, int tid, int nthr) {
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P; i += nthr) {
        int l = i ^ j;
        if (l > i) {
          int32_t a = buf[i], b = buf[l];
          bool up = (i & k) == 0;
          if ((a > b) == up) { buf[i] = b; buf[l] = a; }
        }
      }
      if (kBlock) __syncthreads(); else __syncwarp();
    }
  }
}

// Gather the candidate columns of row i of S (i itself and every row of every
// column of A in row i) into buf, pad to a power of two and sort.  Returns P.
template <bool kBlock>
__device__ int gather_sorted(int64_t i, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const int64_t* __restrict__ trp, const int32_t* __restrict__ tci, int32_t* buf,
                             int cand, int tid, int nthr) {
  int P = 1;
  while (P < cand) P <<= 1;
  if (tid == 0) buf[0] = (int32_t)i;
  int at = 1;
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
    const int32_t k = ci[p];
    const int64_t s = trp[k], len = trp[k + 1] - s;
    for (int64_t q = tid; q < len; q += nthr) buf[at + q] = tci[s + q];
    at += (int)len;
  }
  for (int q = cand + tid; q < P; q += nthr) buf[q] = INT32_MAX;
  if (kBlock) __syncthreads(); else __syncwarp();
  bitonic_sort<kBlock>(buf, P, tid, nthr);
  return P;
}

__device__ __forceinline__ int candidates(int64_t i, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                          const int64_t* __restrict__ trp) {
  int64_t c = 0;
  for (int64_t p = rp[i] + lane_id(); p < rp[i + 1]; p += 32) c += trp[ci[p] + 1] - trp[ci[p]];
  c = warp_sum(c);
  return (int)min(c + 1, (int64_t)INT32_MAX);
}

// Warp per row: count (kFill = false) or write (kFill = true) the sorted
// unique columns of row i of S.  Rows with more than kSymCap candidates are
// appended to `long_rows` for the CTA-per-row kernel.
template <bool kFill>
__global__ void __launch_bounds__(kSetupWarps * 32) k_sym_warp(int64_t m, const int64_t* __restrict__ rp,
                                                               const int32_t* __restrict__ ci,
                                                               const int64_t* __restrict__ trp,
                                                               const int32_t* __restrict__ tci,
                                                               int64_t* __restrict__ srp, int32_t* __restrict__ sci,
                                                               int32_t* __restrict__ long_rows,
                                                               int32_t* __restrict__ nlong) {
  __shared__ int32_t sbuf[kSetupWarps][kSymCap];
  const int w = threadIdx.x >> 5, lane = lane_id();
  int32_t* buf = sbuf[w];
  for (int64_t i = blockIdx.x * (int64_t)kSetupWarps + w; i < m; i += (int64_t)gridDim.x * kSetupWarps) {
    const int cand = candidates(i, rp, ci, trp);
    if (cand > kSymCap) {
      if (!kFill && lane == 0) long_rows[atomicAdd(nlong, 1)] = (int32_t)i;
      continue;
    }
    const int P = gather_sorted<false>(i, rp, ci, trp, tci, buf, cand, lane, 32);
    int64_t out = kFill ? srp[i] : 0;
    for (int base = 0; base < P; base += 32) {
      const int q = base + lane;
      const int32_t c = q < P ? buf[q] : INT32_MAX;  // P may be < 32
      const bool first = c != INT32_MAX && (q == 0 || buf[q - 1] != c);
      const unsigned mask = __ballot_sync(0xffffffffu, first);
      if (kFill && first) sci[out + __popc(mask & ((1u << lane) - 1u))] = c;
      out += __popc(mask);
    }
    if (!kFill && lane == 0) srp[i] = out;
    __syncwarp();
  }
}

// CTA per long row (up to kLongCap candidates, dynamic shared memory).
template <bool kFill>
__global__ void k_sym_long(const int32_t* __restrict__ rows, const int64_t* __restrict__ rp,
                           const int32_t* __restrict__ ci, const int64_t* __restrict__ trp,
                           const int32_t* __restrict__ tci, int64_t* __restrict__ srp, int32_t* __restrict__ sci,
                           int* __restrict__ err) {
  extern __shared__ int32_t dbuf[];
  __shared__ int64_t cnt_sh[33];
  const int64_t i = rows[blockIdx.x];
  int64_t c = 0;
  for (int64_t p = rp[i] + threadIdx.x; p < rp[i + 1]; p += blockDim.x) c += trp[ci[p] + 1] - trp[ci[p]];
  c = warp_sum(c);
  if (lane_id() == 0) cnt_sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 1;
    for (unsigned k = 0; k < blockDim.x / 32; ++k) t += cnt_sh[k];
    cnt_sh[32] = t;
  }
  __syncthreads();
  const int64_t cand = cnt_sh[32];
  if (cand > kLongCap) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  const int P = gather_sorted<true>(i, rp, ci, trp, tci, dbuf, (int)cand, threadIdx.x, blockDim.x);
  __shared__ int64_t run;
  __shared__ int32_t wcnt[32];
  if (threadIdx.x == 0) run = kFill ? srp[i] : 0;
  __syncthreads();
  for (int base = 0; base < P; base += blockDim.x) {
    const int q = base + threadIdx.x;
    const int32_t cc = q < P ? dbuf[q] : INT32_MAX;
    const bool first = cc != INT32_MAX && (q == 0 || dbuf[q - 1] != cc);
    const unsigned mask = __ballot_sync(0xffffffffu, first);
    if (lane_id() == 0) wcnt[threadIdx.x >> 5] = __popc(mask);
    __syncthreads();
    int64_t before = run;
    for (unsigned k = 0; k < (threadIdx.x >> 5); ++k) before += wcnt[k];
    if (kFill && first) sci[before + __popc(mask & ((1u << lane_id()) - 1u))] = cc;
    __syncthreads();
    if (threadIdx.x == 0) {
      int64_t t = 0;
      for (unsigned k = 0; k < blockDim.x / 32; ++k) t += wcnt[k];
      run += t;
    }
    __syncthreads();
  }
  if (!kFill && threadIdx.x == 0) srp[i] = run;
}

// Values of S on its pattern, warp per row; see the rounding rule above.
constexpr int kNumCap = 512;
__global__ void __launch_bounds__(kSetupWarps * 32) k_normal_values(
    int64_t m, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const double* __restrict__ v,
    const int64_t* __restrict__ trp, const int32_t* __restrict__ tci, const double* __restrict__ tv,
    const double* __restrict__ theta, double rho, const int64_t* __restrict__ srp,
    const int32_t* __restrict__ sci, double* __restrict__ sv) {
  __shared__ int32_t scol[kSetupWarps][kNumCap];
  __shared__ double sacc[kSetupWarps][kNumCap];
  const int w = threadIdx.x >> 5, lane = lane_id();
  for (int64_t i = blockIdx.x * (int64_t)kSetupWarps + w; i < m; i += (int64_t)gridDim.x * kSetupWarps) {
    const int64_t s0 = srp[i], len = srp[i + 1] - s0;
    const bool local = len <= kNumCap;
    int32_t* cols = local ? scol[w] : nullptr;
    double* acc = local ? sacc[w] : sv + s0;
    for (int64_t q = lane; q < len; q += 32) {
      if (local) cols[q] = sci[s0 + q];
      acc[q] = 0.0;
    }
    __syncwarp();
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int32_t k = ci[p];
      const double aik = v[p], th = theta[k];
      const double ti = __dmul_rn(aik, th);
      const int64_t cs = trp[k], ce = trp[k + 1];
      for (int64_t q = cs + lane; q < ce; q += 32) {
        const int32_t j = tci[q];
        const double ajk = tv[q];
        const int64_t pos = local ? bsearch_i32(cols, 0, len, j) : bsearch_i32(sci + s0, 0, len, j);
        const double prod = (j <= i) ? __fma_rn(ti, ajk, acc[pos]) : __fma_rn(__dmul_rn(ajk, th), aik, acc[pos]);
        acc[pos] = prod;
      }
      __syncwarp();
    }
    if (lane == 0) {
      const int64_t d = local ? bsearch_i32(cols, 0, len, (int32_t)i) : bsearch_i32(sci + s0, 0, len, (int32_t)i);
      acc[d] = __dadd_rn(acc[d], rho);
    }
    __syncwarp();
    if (local)
      for (int64_t q = lane; q < len; q += 32) sv[s0 + q] = acc[q];
    __syncwarp();
  }
}

// ---------------------------------------------------------------- augmented

// For the augmented form: position of every unknown in the BBD order.
__global__ void k_bbd_positions(int64_t m, int64_t n, int64_t nblocks, const int64_t* __restrict__ rbp,
                                const int64_t* __restrict__ cbp, const int64_t* __restrict__ kbp,
                                int64_t* __restrict__ pos) {
  // x_j of block k -> kbp[k] + (j - cbp[k]); lambda_i of block k -> kbp[k] + n_k + (i - rbp[k]);
  // linking row i -> kbp[nblocks] + (i - rbp[nblocks]).
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n + m; u += (int64_t)gridDim.x * blockDim.x) {
    if (u < n) {
      int64_t lo = 0, hi = nblocks;  // block with cbp[k] <= u < cbp[k+1]
      while (hi - lo > 1) { int64_t mid = (lo + hi) >> 1; if (cbp[mid] <= u) lo = mid; else hi = mid; }
      pos[u] = kbp[lo] + (u - cbp[lo]);
    } else {
      const int64_t i = u - n;
      if (i >= rbp[nblocks]) { pos[u] = kbp[nblocks] + (i - rbp[nblocks]); continue; }
      int64_t lo = 0, hi = nblocks;
      while (hi - lo > 1) { int64_t mid = (lo + hi) >> 1; if (rbp[mid] <= i) lo = mid; else hi = mid; }
      pos[u] = kbp[lo] + (cbp[lo + 1] - cbp[lo]) + (i - rbp[lo]);
    }
  }
}

__global__ void k_aug_count(int64_t m, int64_t n, const int64_t* __restrict__ rp, const int64_t* __restrict__ trp,
                            const int64_t* __restrict__ pos, int64_t* __restrict__ krp) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n + m; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cnt = u < n ? 1 + trp[u + 1] - trp[u] : 1 + rp[u - n + 1] - rp[u - n];
    krp[pos[u]] = cnt;
  }
}

// Row of K for unknown u (new index pos[u]), written unsorted, then sorted by
// k_sort_segments.  x_u: diagonal fl(-1/theta_u) and column u of A; lambda_i:
// row i of A and the diagonal rho.
__global__ void k_aug_fill(int64_t m, int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, const int64_t* __restrict__ trp,
                           const int32_t* __restrict__ tci, const double* __restrict__ tv,
                           const double* __restrict__ theta, double rho, const int64_t* __restrict__ pos,
                           const int64_t* __restrict__ krp, int32_t* __restrict__ kci, double* __restrict__ kv) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n + m; u += (int64_t)gridDim.x * blockDim.x) {
    int64_t at = krp[pos[u]];
    if (u < n) {
      kci[at] = (int32_t)pos[u];
      kv[at++] = __ddiv_rn(-1.0, theta[u]);
      for (int64_t q = trp[u]; q < trp[u + 1]; ++q) { kci[at] = (int32_t)pos[n + tci[q]]; kv[at++] = tv[q]; }
    } else {
      const int64_t i = u - n;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) { kci[at] = (int32_t)pos[ci[p]]; kv[at++] = v[p]; }
      kci[at] = (int32_t)pos[u];
      kv[at] = rho;
    }
  }
}

// New theta for the augmented form: only the x diagonal entries change.
__global__ void k_aug_theta(int64_t n, const double* __restrict__ theta, const int64_t* __restrict__ xdiag,
                            double* __restrict__ kv) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    kv[xdiag[u]] = __ddiv_rn(-1.0, theta[u]);
}

__global__ void k_aug_xdiag(int64_t n, const int64_t* __restrict__ pos, const int64_t* __restrict__ krp,
                            const int32_t* __restrict__ kci, int64_t* __restrict__ xdiag) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = pos[u];
    xdiag[u] = bsearch_i32(kci, krp[r], krp[r + 1], (int32_t)r);
  }
}

// CSR validity: row pointers non-decreasing, columns in range and strictly
// ascending inside every row.  Sets *bad on the first violation.
__global__ void k_check_csr(int64_t nrows, int64_t ncols, const int64_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, int* __restrict__ bad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = rp[i], e = rp[i + 1];
    if (e < s) { atomicExch(bad, 1); continue; }
    for (int64_t p = s; p < e; ++p) {
      const int32_t c = ci[p];
      if (c < 0 || c >= ncols || (p > s && ci[p - 1] >= c)) { atomicExch(bad, 1); break; }
    }
  }
}

inline unsigned grid_for(int64_t work, int per_block, int cap = 152 * 32) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

}  // namespace

cudaError_t check_csr(int64_t nrows, int64_t ncols, const int64_t* rp, const int32_t* ci, int* bad,
                      cudaStream_t st) {
  k_check_csr<<<grid_for(nrows, 256), 256, 0, st>>>(nrows, ncols, rp, ci, bad); count_launch();
  return cudaGetLastError();
}

cudaError_t transpose_csr(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v, int64_t* trp,
                          int32_t* tci, double* tv, int64_t* scan_scratch, cudaStream_t st) {
  SDSL_CUDA_TRY(cudaMemsetAsync(trp, 0, sizeof(int64_t) * (size_t)(n + 1), st));
  k_transpose_count<<<grid_for(m, 256), 256, 0, st>>>(m, rp, ci, reinterpret_cast<unsigned long long*>(trp)); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  SDSL_CUDA_TRY(exclusive_scan_i64(trp, n, scan_scratch, st));
  // cursor: reuse the scan scratch? it is small; use tci's neighbour buffer from the caller instead
  return cudaSuccess;
}

cudaError_t transpose_fill(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                           const int64_t* trp, int32_t* tci, double* tv, int64_t* cursor, cudaStream_t st) {
  SDSL_CUDA_TRY(cudaMemcpyAsync(cursor, trp, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
  k_transpose_fill<<<grid_for(m, 256), 256, 0, st>>>(m, rp, ci, v, reinterpret_cast<unsigned long long*>(cursor),
                                                     tci, tv); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  k_sort_segments<<<grid_for(n, 256), 256, 0, st>>>(n, trp, tci, tv); count_launch();
  return cudaGetLastError();
}

cudaError_t sort_rows(int64_t nrows, const int64_t* rp, int32_t* ci, double* v, cudaStream_t st) {
  k_sort_segments<<<grid_for(nrows, 256), 256, 0, st>>>(nrows, rp, ci, v); count_launch();
  return cudaGetLastError();
}

cudaError_t normal_symbolic_count(int64_t m, const int64_t* rp, const int32_t* ci, const int64_t* trp,
                                  const int32_t* tci, int64_t* srp, int32_t* long_rows, int32_t* nlong,
                                  cudaStream_t st) {
  SDSL_CUDA_TRY(cudaMemsetAsync(nlong, 0, sizeof(int32_t), st));
  k_sym_warp<false><<<grid_for(m, kSetupWarps), kSetupWarps * 32, 0, st>>>(m, rp, ci, trp, tci, srp, nullptr,
                                                                           long_rows, nlong); count_launch();
  return cudaGetLastError();
}

cudaError_t normal_symbolic_long(bool fill, int nlong, const int32_t* long_rows, const int64_t* rp,
                                 const int32_t* ci, const int64_t* trp, const int32_t* tci, int64_t* srp,
                                 int32_t* sci, int* err, cudaStream_t st) {
  if (nlong == 0) return cudaSuccess;
  const size_t smem = sizeof(int32_t) * kLongCap;
  if (fill) {
    SDSL_CUDA_TRY((allow_max_dynamic_smem<k_sym_long<true>>()));
    k_sym_long<true><<<nlong, 1024, smem, st>>>(long_rows, rp, ci, trp, tci, srp, sci, err); count_launch();
  } else {
    SDSL_CUDA_TRY((allow_max_dynamic_smem<k_sym_long<false>>()));
    k_sym_long<false><<<nlong, 1024, smem, st>>>(long_rows, rp, ci, trp, tci, srp, sci, err); count_launch();
  }
  return cudaGetLastError();
}

cudaError_t normal_symbolic_fill(int64_t m, const int64_t* rp, const int32_t* ci, const int64_t* trp,
                                 const int32_t* tci, const int64_t* srp, int32_t* sci, cudaStream_t st) {
  k_sym_warp<true><<<grid_for(m, kSetupWarps), kSetupWarps * 32, 0, st>>>(m, rp, ci, trp, tci,
                                                                          const_cast<int64_t*>(srp), sci, nullptr,
                                                                          nullptr); count_launch();
  return cudaGetLastError();
}

cudaError_t normal_values(int64_t m, const int64_t* rp, const int32_t* ci, const double* v, const int64_t* trp,
                          const int32_t* tci, const double* tv, const double* theta, double rho,
                          const int64_t* srp, const int32_t* sci, double* sv, cudaStream_t st) {
  k_normal_values<<<grid_for(m, kSetupWarps), kSetupWarps * 32, 0, st>>>(m, rp, ci, v, trp, tci, tv, theta, rho, srp,
                                                                         sci, sv); count_launch();
  return cudaGetLastError();
}

cudaError_t bbd_positions(int64_t m, int64_t n, int64_t nblocks, const int64_t* rbp, const int64_t* cbp,
                          const int64_t* kbp, int64_t* pos, cudaStream_t st) {
  k_bbd_positions<<<grid_for(n + m, 256), 256, 0, st>>>(m, n, nblocks, rbp, cbp, kbp, pos); count_launch();
  return cudaGetLastError();
}

cudaError_t augmented_count(int64_t m, int64_t n, const int64_t* rp, const int64_t* trp, const int64_t* pos,
                            int64_t* krp, cudaStream_t st) {
  k_aug_count<<<grid_for(n + m, 256), 256, 0, st>>>(m, n, rp, trp, pos, krp); count_launch();
  return cudaGetLastError();
}

cudaError_t augmented_fill(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                           const int64_t* trp, const int32_t* tci, const double* tv, const double* theta, double rho,
                           const int64_t* pos, const int64_t* krp, int32_t* kci, double* kv, int64_t* xdiag,
                           cudaStream_t st) {
  k_aug_fill<<<grid_for(n + m, 256), 256, 0, st>>>(m, n, rp, ci, v, trp, tci, tv, theta, rho, pos, krp, kci, kv); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  k_sort_segments<<<grid_for(n + m, 256), 256, 0, st>>>(n + m, krp, kci, kv); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  k_aug_xdiag<<<grid_for(n, 256), 256, 0, st>>>(n, pos, krp, kci, xdiag); count_launch();
  return cudaGetLastError();
}

cudaError_t augmented_theta(int64_t n, const double* theta, const int64_t* xdiag, double* kv, cudaStream_t st) {
  k_aug_theta<<<grid_for(n, 256), 256, 0, st>>>(n, theta, xdiag, kv); count_launch();
  return cudaGetLastError();
}

}  // namespace sdsl
