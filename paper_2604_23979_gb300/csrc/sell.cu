// sell.cu -- sliced ELL (SELL-32) copies of A and A^T for the factored
// normal-equation product S p = A (theta o (A^T p)) + rho p (Eq. (schur)).
//
// Rows are ranked by length (longest first, then by index) inside windows of
// kWindow rows; every 32 consecutive ranked rows form a slice whose entries
// are stored slot-major (entry j of the slice's 32 rows contiguous), padded to
// the slice's longest row with column -1.  One warp takes a slice, a lane a
// row: no row-pointer round trip, and every entry load is one coalesced line.
// The product value of ranked row r is written to its original row perm[r].
#include <algorithm>

#include "pcg_common.cuh"

namespace sdsl {

namespace {

constexpr int kWindow = 256;
constexpr int kSellThreads = 256;

// Rank the rows of each window by (length descending, index ascending).
__global__ void __launch_bounds__(kWindow) k_sell_rank(int64_t nrows, const int64_t* __restrict__ rp,
                                                      int32_t* __restrict__ perm) {
  __shared__ int32_t len[kWindow];
  const int64_t w0 = (int64_t)blockIdx.x * kWindow;
  const int64_t i = w0 + threadIdx.x;
  const int nw = (int)(nrows - w0 < kWindow ? nrows - w0 : kWindow);
  len[threadIdx.x] = i < nrows ? (int32_t)(rp[i + 1] - rp[i]) : -1;
  __syncthreads();
  if (i >= nrows) return;
  const int32_t li = len[threadIdx.x];
  int rank = 0;
  for (int j = 0; j < nw; ++j) {
    const int32_t lj = len[j];
    rank += (lj > li || (lj == li && j < (int)threadIdx.x)) ? 1 : 0;
  }
  perm[w0 + rank] = (int32_t)i;
}

// Slice widths (entries x 32 per slice, to be scanned into offsets).
__global__ void k_sell_width(int64_t nrows, int64_t nslices, const int64_t* __restrict__ rp,
                             const int32_t* __restrict__ perm, int32_t* __restrict__ wid, int64_t* __restrict__ cnt) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nslices; s += (int64_t)gridDim.x * blockDim.x) {
    // the longest row of a slice: rows are ranked within windows, and slices
    // never straddle a window (kWindow is a multiple of 32)
    int32_t w = 0;
    for (int k = 0; k < 32; ++k) {
      const int64_t r = s * 32 + k;
      if (r < nrows) {
        const int64_t row = perm[r];
        w = max(w, (int32_t)(rp[row + 1] - rp[row]));
      }
    }
    wid[s] = w;
    cnt[s] = (int64_t)w * 32;
  }
}

__global__ void k_sell_fill(int64_t nrows, int64_t nslices, const int64_t* __restrict__ rp,
                            const int32_t* __restrict__ ci, const double* __restrict__ v,
                            const int32_t* __restrict__ perm, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ wid, int32_t* __restrict__ scol, double* __restrict__ sval) {
  const int lane = lane_id();
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t s = warp; s < nslices; s += nwarps) {
    const int64_t r = s * 32 + lane;
    int64_t a = 0, len = 0;
    if (r < nrows) {
      const int64_t row = perm[r];
      a = rp[row];
      len = rp[row + 1] - a;
    }
    const int64_t base = off[s];
    for (int32_t j = 0; j < wid[s]; ++j) {
      const bool ok = j < len;
      scol[base + (int64_t)j * 32 + lane] = ok ? ci[a + j] : -1;
      sval[base + (int64_t)j * 32 + lane] = ok ? v[a + j] : 0.0;
    }
  }
}

// Row value of the lane's ranked row: four independent accumulators over the
// slice's slots (padding, column -1, is skipped).
__device__ __forceinline__ double sell_row(const SellMat& S, int64_t s, const double* __restrict__ x) {
  const int lane = lane_id();
  const int64_t base = S.off[s];
  const int32_t w = S.wid[s];
  const int32_t* __restrict__ col = S.col + base + lane;
  const double* __restrict__ val = S.val + base + lane;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int32_t j = 0;
  for (; j + 3 < w; j += 4) {
    const int32_t c0 = __ldcs(col + 32 * j), c1 = __ldcs(col + 32 * (j + 1)), c2 = __ldcs(col + 32 * (j + 2)),
                  c3 = __ldcs(col + 32 * (j + 3));
    const double v0 = __ldcs(val + 32 * j), v1 = __ldcs(val + 32 * (j + 1)), v2 = __ldcs(val + 32 * (j + 2)),
                 v3 = __ldcs(val + 32 * (j + 3));
    if (c0 >= 0) a0 = __fma_rn(v0, __ldg(x + c0), a0);
    if (c1 >= 0) a1 = __fma_rn(v1, __ldg(x + c1), a1);
    if (c2 >= 0) a2 = __fma_rn(v2, __ldg(x + c2), a2);
    if (c3 >= 0) a3 = __fma_rn(v3, __ldg(x + c3), a3);
  }
  for (; j < w; ++j) {
    const int32_t c = __ldcs(col + 32 * j);
    if (c >= 0) a0 = __fma_rn(__ldcs(val + 32 * j), __ldg(x + c), a0);
  }
  return (a0 + a1) + (a2 + a3);
}

// u = theta o (A^T p) on the SELL copy of A^T; (vb, vg): this CTA's index
// and the grid it belongs to (a request's virtual grid in a batched launch).
__device__ __forceinline__ void sell_at_theta_body(const SellMat& S, const double* __restrict__ theta,
                                                   const double* __restrict__ p, double* __restrict__ u, int vb,
                                                   int vg) {
  const int lane = lane_id();
  const int64_t warp = ((int64_t)vb * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)vg * blockDim.x) >> 5;
  for (int64_t sl = warp; sl < S.nslices; sl += nwarps) {
    const double acc = sell_row(S, sl, p);
    const int64_t r = sl * 32 + lane;
    if (r < S.nrows) {
      const int64_t k = S.perm[r];
      u[k] = theta[k] * acc;
    }
  }
}

__global__ void __launch_bounds__(kSellThreads) k_sell_at_theta(SellMat S, const double* __restrict__ theta,
                                                               const double* __restrict__ p, double* __restrict__ u,
                                                               const PcgState* __restrict__ s) {
  if (s && s->done) return;
  sell_at_theta_body(S, theta, p, u, (int)blockIdx.x, (int)gridDim.x);
}

// q = A u + rho p on the SELL copy of A; with pcg 1: partial p^T q per CTA, the
// last CTA of the grid sums the partials in CTA order and sets alpha, iters;
// pcg 2: the product alone, skipped once the solve has stopped.
__device__ __forceinline__ void sell_a_u_dot_body(const SellMat& S, const double* __restrict__ u, double rho,
                                                  const double* __restrict__ p, double* __restrict__ q,
                                                  double* __restrict__ part, PcgState* __restrict__ s, int pcg,
                                                  int vb, int vg) {
  __shared__ double sh[kSellThreads / 32];
  const int lane = lane_id();
  const int64_t warp = ((int64_t)vb * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)vg * blockDim.x) >> 5;
  double loc = 0.0;
  for (int64_t sl = warp; sl < S.nslices; sl += nwarps) {
    const double acc = sell_row(S, sl, u);
    const int64_t r = sl * 32 + lane;
    if (r < S.nrows) {
      const int64_t i = S.perm[r];
      const double qi = __fma_rn(rho, p[i], acc);
      q[i] = qi;
      loc = __fma_rn(p[i], qi, loc);
    }
  }
  if (pcg != 1) return;
  const double tot = block_sum(loc, sh);
  if (threadIdx.x == 0) part[vb] = tot;
  if (last_block(&s->ticket[0], (unsigned)vg)) {
    if (threadIdx.x < 32) {
      const double pq = warp_fixed_sum(part, vg);
      if (threadIdx.x == 0) {
        s->pq = pq;
        s->alpha = s->rho / pq;
        s->iters += 1;
        if (!(pq > 0.0) || !isfinite(pq)) s->done = 3;
        s->ticket[0] = 0;
      }
    }
  }
}

__global__ void __launch_bounds__(kSellThreads) k_sell_a_u_dot(SellMat S, const double* __restrict__ u, double rho,
                                                              const double* __restrict__ p, double* __restrict__ q,
                                                              double* __restrict__ part, PcgState* __restrict__ s,
                                                              int pcg) {
  if (pcg && s->done) return;
  sell_a_u_dot_body(S, u, rho, p, q, part, s, pcg, (int)blockIdx.x, (int)gridDim.x);
}

inline unsigned sell_grid(int64_t nslices, int max_ctas) {
  int64_t g = (nslices + kSellThreads / 32 - 1) / (kSellThreads / 32);
  if (g > max_ctas) g = max_ctas;
  return (unsigned)(g < 1 ? 1 : g);
}

// The two halves of the factored product over several requests, one
// persistent launch each: items (request, virtual CTA) of each request's own
// grid, so every request's partial sums and ticket are those of its single
// launch.
__global__ void __launch_bounds__(kSellThreads) k_batch_sell_at_theta(const BatchReq* __restrict__ reqs,
                                                                     const BatchItem* __restrict__ items, int nitems) {
  __shared__ int skip;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem I = items[it];
    const BatchReq& R = reqs[I.req];
    __syncthreads();
    if (threadIdx.x == 0) skip = R.s->done;
    __syncthreads();
    if (skip) continue;
    sell_at_theta_body(R.A.at_sell, R.A.theta, R.p, R.A.u, I.vb, R.g_at);
  }
}

__global__ void __launch_bounds__(kSellThreads) k_batch_sell_a_u_dot(const BatchReq* __restrict__ reqs,
                                                                    const BatchItem* __restrict__ items, int nitems) {
  __shared__ int skip;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem I = items[it];
    const BatchReq& R = reqs[I.req];
    __syncthreads();
    if (threadIdx.x == 0) skip = R.s->done;
    __syncthreads();
    if (skip) continue;
    sell_a_u_dot_body(R.A.a_sell, R.A.u, R.A.rho, R.p, R.q, R.part, R.s, 1, I.vb, R.g_a);
  }
}

}  // namespace

int sell_occupancy(int which) {
  int n = 0;
  if (which == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sell_at_theta, kSellThreads, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sell_a_u_dot, kSellThreads, 0);
  return n > 0 ? n : 1;
}

cudaError_t sell_rank_widths(int64_t nrows, const int64_t* rp, int32_t* perm, int32_t* wid, int64_t* cnt,
                             cudaStream_t st) {
  const int64_t nslices = (nrows + 31) / 32;
  if (nrows == 0) return cudaSuccess;
  k_sell_rank<<<(unsigned)((nrows + kWindow - 1) / kWindow), kWindow, 0, st>>>(nrows, rp, perm); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  k_sell_width<<<(unsigned)std::min<int64_t>((nslices + 255) / 256, 152 * 16), 256, 0, st>>>(nrows, nslices, rp,
                                                                                              perm, wid, cnt); count_launch();
  return cudaGetLastError();
}

cudaError_t sell_fill(int64_t nrows, const int64_t* rp, const int32_t* ci, const double* v, const int32_t* perm,
                      const int64_t* off, const int32_t* wid, int32_t* col, double* val, cudaStream_t st) {
  const int64_t nslices = (nrows + 31) / 32;
  if (nslices == 0) return cudaSuccess;
  k_sell_fill<<<(unsigned)std::min<int64_t>((nslices + 7) / 8, 152 * 16), 256, 0, st>>>(nrows, nslices, rp, ci, v,
                                                                                         perm, off, wid, col, val); count_launch();
  return cudaGetLastError();
}

cudaError_t sell_factored_product(const SpmvPlan& A, const double* p, double* q, double* part, PcgState* s, int pcg,
                                  cudaStream_t st) {
  k_sell_at_theta<<<A.sell_at_grid, kSellThreads, 0, st>>>(A.at_sell, A.theta, p, A.u, pcg ? s : nullptr); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  k_sell_a_u_dot<<<A.sell_a_grid, kSellThreads, 0, st>>>(A.a_sell, A.u, A.rho, p, q, part, s, pcg); count_launch();
  return cudaGetLastError();
}

unsigned sell_grid_for(int64_t nslices, int max_ctas) { return sell_grid(nslices, max_ctas); }

cudaError_t batch_product(const BatchReq* reqs, const BatchItem* items_at, int n_at, const BatchItem* items_a,
                          int n_a, int grid, cudaStream_t st) {
  if (n_at > 0) {
    k_batch_sell_at_theta<<<(unsigned)std::min(grid, n_at), kSellThreads, 0, st>>>(reqs, items_at, n_at);
    count_launch();
    SDSL_CUDA_TRY(cudaGetLastError());
  }
  if (n_a > 0) {
    k_batch_sell_a_u_dot<<<(unsigned)std::min(grid, n_a), kSellThreads, 0, st>>>(reqs, items_a, n_a);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace sdsl
