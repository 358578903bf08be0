// bbd.cu -- bordered block-diagonal (BBD) preconditioner and GMRES kernels
// (Sec. 2.4; right preconditioning of Sec. 2.2).
//
// The preconditioner matrix P (filtered, corrected K) is in BBD order:
// interior blocks [bp[k], bp[k+1]), border rows/cols [b0, N), b0 = bp[nb].
// Block factors are ILU(0) on P's layout (unit L at j < i, U at j >= i).
//   Schur complement   S_B = C - sum_k F_k (L_k U_k)^{-1} E_k        (FP64)
//   dense LU of S_B    partial pivoting, FP32 factors; the explicit inverse
//                      S_B^{-1} = U^{-1} L^{-1} P is formed once, so every
//                      application is a dense matrix-vector product
//   apply              y_k = L_k^{-1} r_k;  t_k = U_k^{-1} y_k;
//                      g = r_B - sum_k F_k t_k;  z_B = S_B^{-1} g (FP32 inverse
//                      + FP64 iterative refinement against the FP64 S_B);
//                      z_k = U_k^{-1} L_k^{-1} (r_k - E_k z_B)
// The paper's MPI_Reduce of the Schur parts to process 1 becomes an
// on-device accumulation (blocks processed in order: deterministic), and its
// send/broadcast around the border solve become stream order.
#include "common.cuh"
#include "kernels.cuh"

namespace sdsl {

namespace {

constexpr int kR = 32;  // border columns per Schur tile (one per lane)

inline unsigned grid_for(int64_t work, int per_block, int cap = 152 * 32) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

// S_B = C (the border-border entries of P), row-major nb x nb.
__global__ void k_schur_init(int64_t nb, int64_t b0, const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                             const double* __restrict__ pv, double* __restrict__ SB) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nb; r += (int64_t)gridDim.x * blockDim.x)
    for (int64_t t = prp[b0 + r]; t < prp[b0 + r + 1]; ++t)
      if (pci[t] >= b0) SB[r * nb + (pci[t] - b0)] = pv[t];
}

// One CTA per (tile of kR border columns [c0, c0+kR), block k of the wave):
//   X = E_k[:, tile]  ->  X = U_k^{-1} L_k^{-1} X  ->  C_k[:, tile] = F_k X.
// X is the block's rows x kR (row-major, one column per lane) in scratch;
// C_k is the block's own dense nb x nb contribution (subtracted from S_B in
// block order by k_schur_reduce, the same order as one block at a time).
__global__ void k_schur_wave(const SchurJob* __restrict__ jobs, int64_t b0, int64_t nb,
                             const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                             const double* __restrict__ pv, const double* __restrict__ F,
                             const double* __restrict__ dinv, const int64_t* __restrict__ pdiag,
                             const int32_t* __restrict__ lev_ptr_lo, const int32_t* __restrict__ lev_rows_lo,
                             const int32_t* __restrict__ lev_ptr_up, const int32_t* __restrict__ lev_rows_up,
                             double* __restrict__ Xall, double* __restrict__ Cpart) {
  const SchurJob J = jobs[blockIdx.y];
  const int64_t s = J.s, e = J.e;
  const int64_t c0 = (int64_t)blockIdx.x * kR;
  double* X = Xall + J.xoff + (int64_t)blockIdx.x * (e - s) * kR;
  double* C = Cpart + (int64_t)blockIdx.y * nb * nb;
  const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t c = c0 + lane;
  // scatter E_k[:, tile]
  for (int64_t i = s + w; i < e; i += nw) {
    double v = 0.0;
    if (c < nb) {
      const int64_t q = bsearch_i32(pci, pdiag[i] + 1, prp[i + 1], (int32_t)(b0 + c));
      if (q >= 0) v = pv[q];
    }
    X[(i - s) * kR + lane] = v;
  }
  __syncthreads();
  // forward, unit lower, level by level
  for (int32_t L = J.L0; L < J.L1; ++L) {
    for (int32_t q = lev_ptr_lo[L] + w; q < lev_ptr_lo[L + 1]; q += nw) {
      const int64_t i = lev_rows_lo[q];
      double acc = X[(i - s) * kR + lane];
      for (int64_t t = prp[i]; t < pdiag[i]; ++t) {
        const int64_t j = pci[t];
        if (j >= s) acc = __fma_rn(-F[t], X[(j - s) * kR + lane], acc);
      }
      X[(i - s) * kR + lane] = acc;
    }
    __syncthreads();
  }
  // backward with U (in-block columns only)
  for (int32_t L = J.U0; L < J.U1; ++L) {
    for (int32_t q = lev_ptr_up[L] + w; q < lev_ptr_up[L + 1]; q += nw) {
      const int64_t i = lev_rows_up[q];
      double acc = X[(i - s) * kR + lane];
      for (int64_t t = pdiag[i] + 1; t < prp[i + 1]; ++t) {
        const int64_t j = pci[t];
        if (j < e) acc = __fma_rn(-F[t], X[(j - s) * kR + lane], acc);
      }
      X[(i - s) * kR + lane] = acc * dinv[i];
    }
    __syncthreads();
  }
  // C_k[:, tile] = F_k X   (border rows, block-k columns).  A border row
  // spans every block; its columns are sorted, so only the block's range is
  // visited (first in-block entry by binary search).
  for (int64_t r = w; r < nb; r += nw) {
    double acc = 0.0;
    const int64_t t1 = prp[b0 + r + 1];
    for (int64_t t = lower_bound_i32(pci, prp[b0 + r], t1, (int32_t)s); t < t1; ++t) {
      const int64_t j = pci[t];
      if (j >= e) break;
      acc = __fma_rn(pv[t], X[(j - s) * kR + lane], acc);
    }
    if (c < nb) C[r * nb + c] = acc;
  }
}

// S_B -= C_0, C_1, ... in the wave's block order (element-wise).
__global__ void k_schur_reduce(int64_t nb, int nk, const double* __restrict__ Cpart, double* __restrict__ SB) {
  const int64_t tot = nb * nb;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    double v = SB[i];
    for (int k = 0; k < nk; ++k) v -= Cpart[(int64_t)k * tot + i];
    SB[i] = v;
  }
}

// ---------------------------------------------------------------- dense LU (FP32)

__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// Step k of right-looking LU: pivot = largest |a_ik|, i >= k (lowest i on
// ties), swap rows k and p, record ipiv[k].  One CTA.
__global__ void k_lu_pivot(int64_t n, int64_t k, float* __restrict__ A, int32_t* __restrict__ ipiv,
                           int* __restrict__ status) {
  __shared__ float bv[32];
  __shared__ int64_t bi[32];
  float best = -1.f;
  int64_t bidx = k;
  for (int64_t i = k + threadIdx.x; i < n; i += blockDim.x) {
    const float v = fabsf(A[i * n + k]);
    if (v > best) { best = v; bidx = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
  }
  if (lane_id() == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = bidx; }
  __syncthreads();
  __shared__ int64_t piv;
  if (threadIdx.x == 0) {
    float b = -1.f;
    int64_t p = k;
    for (unsigned w = 0; w < blockDim.x / 32; ++w)
      if (bv[w] > b || (bv[w] == b && bi[w] < p)) { b = bv[w]; p = bi[w]; }
    piv = p;
    ipiv[k] = (int32_t)p;
    if (!(b > 0.f) || !isfinite(b)) *status = 1;
  }
  __syncthreads();
  const int64_t p = piv;
  if (p != k)
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
      const float t = A[k * n + j];
      A[k * n + j] = A[p * n + j];
      A[p * n + j] = t;
    }
}

// Rows i > k: l_ik = a_ik / a_kk; a_ij -= l_ik a_kj for j > k.
__global__ void k_lu_update(int64_t n, int64_t k, float* __restrict__ A) {
  const float piv = A[k * n + k];
  for (int64_t i = k + 1 + blockIdx.x; i < n; i += gridDim.x) {
    const float l = A[i * n + k] / piv;
    for (int64_t j = k + 1 + threadIdx.x; j < n; j += blockDim.x) A[i * n + j] = __fmaf_rn(-l, A[k * n + j], A[i * n + j]);
    __syncthreads();
    if (threadIdx.x == 0) A[i * n + k] = l;
  }
}

// Inverse from the LU factors: column c of X solves L U x = e_{perm(c)}.
// One CTA per 32 columns (one per lane), rows swept in order.
__global__ void k_lu_inverse(int64_t n, const float* __restrict__ LU, const int32_t* __restrict__ ipiv,
                             float* __restrict__ Xinv, float* __restrict__ work) {
  const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t c = (int64_t)blockIdx.x * 32 + lane;
  float* x = work + (int64_t)blockIdx.x * n * 32;  // n x 32 column tile, row-major
  // b = P e_c: apply the row swaps to the identity column
  for (int64_t i = w; i < n; i += nw) x[i * 32 + lane] = (i == c) ? 1.f : 0.f;
  __syncthreads();
  if (w == 0) {
    for (int64_t k = 0; k < n; ++k) {
      const int64_t p = ipiv[k];
      if (p != k) {
        const float t = x[k * 32 + lane];
        x[k * 32 + lane] = x[p * 32 + lane];
        x[p * 32 + lane] = t;
      }
    }
  }
  __syncthreads();
  // forward (unit L), column-oriented with all warps splitting the trailing rows
  for (int64_t k = 0; k < n; ++k) {
    const float xk = x[k * 32 + lane];
    for (int64_t i = k + 1 + w; i < n; i += nw) x[i * 32 + lane] = __fmaf_rn(-LU[i * n + k], xk, x[i * 32 + lane]);
    __syncthreads();
  }
  for (int64_t k = n - 1; k >= 0; --k) {
    if (w == 0) x[k * 32 + lane] = x[k * 32 + lane] / LU[k * n + k];
    __syncthreads();
    const float xk = x[k * 32 + lane];
    for (int64_t i = w; i < k; i += nw) x[i * 32 + lane] = __fmaf_rn(-LU[i * n + k], xk, x[i * 32 + lane]);
    __syncthreads();
  }
  if (c < n)
    for (int64_t i = w; i < n; i += nw) Xinv[i * n + c] = x[i * 32 + lane];
}

// ---------------------------------------------------------------- BBD apply

// Block LU solves y_k = U_k^{-1} L_k^{-1} y_k for every interior block (one
// CTA per block), level by level.  A row is summed by a group of kLuV lanes
// (rows here have tens of entries); the loop over a level's rows is
// warp-uniform so the group shuffles see every lane.
constexpr int kLuV = 4;
__global__ void k_block_lu_solve(const int64_t* __restrict__ bp, const int64_t* __restrict__ prp,
                                 const int32_t* __restrict__ pci, const double* __restrict__ F,
                                 const double* __restrict__ dinv, const int64_t* __restrict__ pdiag,
                                 const int32_t* __restrict__ lev_off_lo, const int32_t* __restrict__ lev_ptr_lo,
                                 const int32_t* __restrict__ lev_rows_lo, const int32_t* __restrict__ lev_off_up,
                                 const int32_t* __restrict__ lev_ptr_up, const int32_t* __restrict__ lev_rows_up,
                                 double* __restrict__ y) {
  const int b = blockIdx.x;
  const int64_t s = bp[b], e = bp[b + 1];
  const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int g = lane / kLuV, sub = lane % kLuV;
  constexpr int kRows = 32 / kLuV;  // rows per warp step
  for (int32_t L = lev_off_lo[b]; L < lev_off_lo[b + 1]; ++L) {
    const int32_t q0 = lev_ptr_lo[L], q1 = lev_ptr_lo[L + 1];
    for (int32_t base = q0 + w * kRows; base < q1; base += nw * kRows) {
      const int32_t q = base + g;
      const bool valid = q < q1;
      const int64_t i = valid ? lev_rows_lo[q] : 0;
      double acc = 0.0;
      if (valid)
        for (int64_t t = prp[i] + sub; t < pdiag[i]; t += kLuV) {
          const int64_t j = pci[t];
          if (j >= s) acc = __fma_rn(F[t], y[j], acc);
        }
      acc = group_sum<kLuV>(acc);
      if (valid && sub == 0) y[i] -= acc;
    }
    __syncthreads();
  }
  for (int32_t L = lev_off_up[b]; L < lev_off_up[b + 1]; ++L) {
    const int32_t q0 = lev_ptr_up[L], q1 = lev_ptr_up[L + 1];
    for (int32_t base = q0 + w * kRows; base < q1; base += nw * kRows) {
      const int32_t q = base + g;
      const bool valid = q < q1;
      const int64_t i = valid ? lev_rows_up[q] : 0;
      double acc = 0.0;
      if (valid)
        for (int64_t t = pdiag[i] + 1 + sub; t < prp[i + 1]; t += kLuV) {
          const int64_t j = pci[t];
          if (j >= e) break;  // columns are sorted: the rest lie beyond the block
          acc = __fma_rn(F[t], y[j], acc);
        }
      acc = group_sum<kLuV>(acc);
      if (valid && sub == 0) y[i] = (y[i] - acc) * dinv[i];
    }
    __syncthreads();
  }
}

// g = r_B - sum over interior columns of P[border rows] t   (warp per border row)
__global__ void k_border_gather(int64_t nb, int64_t b0, const int64_t* __restrict__ prp,
                                const int32_t* __restrict__ pci, const double* __restrict__ pv,
                                const double* __restrict__ r, const double* __restrict__ t, double* __restrict__ g) {
  const int lane = lane_id();
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = wid; row < nb; row += nwarps) {
    double acc = 0.0;
    for (int64_t q = prp[b0 + row] + lane; q < prp[b0 + row + 1]; q += 32) {
      const int64_t j = pci[q];
      if (j < b0) acc = __fma_rn(pv[q], t[j], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) g[row] = r[b0 + row] - acc;
  }
}

// w_i = r_i - sum over border columns of P[i, border] z_B, interior rows
__global__ void k_border_scatter(int64_t b0, const int64_t* __restrict__ prp, const int32_t* __restrict__ pci,
                                 const int64_t* __restrict__ pdiag, const double* __restrict__ pv,
                                 const double* __restrict__ r, const double* __restrict__ zB,
                                 double* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b0; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = r[i];
    for (int64_t q = pdiag[i] + 1; q < prp[i + 1]; ++q) {
      const int64_t j = pci[q];
      if (j >= b0) acc = __fma_rn(-pv[q], zB[j - b0], acc);
    }
    w[i] = acc;
  }
}

// y = A x for a dense row-major n x n FP32 (mode 0) or FP64 (mode 1) matrix;
// mode 2: y = b - A x with FP64 A (refinement residual).  Warp per row.
template <typename T>
__global__ void k_dense_mv(int64_t n, const T* __restrict__ A, const double* __restrict__ x,
                           const double* __restrict__ b, double* __restrict__ y, int residual) {
  const int lane = lane_id();
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = wid; i < n; i += nwarps) {
    double acc = 0.0;
    for (int64_t j = lane; j < n; j += 32) acc = __fma_rn((double)A[i * n + j], x[j], acc);
    acc = warp_sum(acc);
    if (lane == 0) y[i] = residual ? b[i] - acc : acc;
  }
}

__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __fma_rn(a, x[i], y[i]);
}

__global__ void k_copy_range(int64_t n, const double* __restrict__ a, double* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// ---------------------------------------------------------------- GMRES helpers

// Partial dot products of w with basis vectors V[0..nv) (each length n,
// stride ldv): part[i * G + cta]; deterministic for a fixed grid.
__global__ void k_multidot(int64_t n, int nv, const double* __restrict__ V, int64_t ldv,
                           const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double sh[32];
  for (int i = 0; i < nv; ++i) {
    double loc = 0.0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
      loc = __fma_rn(V[i * ldv + k], w[k], loc);
    const double t = block_sum(loc, sh);
    if (threadIdx.x == 0) part[(int64_t)i * gridDim.x + blockIdx.x] = t;
    __syncthreads();
  }
}

// One step of modified Gram-Schmidt, fused: w -= hprev * vprev (if vprev),
// then the partial products of the updated w with vcur (or with itself when
// vcur is NULL: the norm of the final w).  part[cta], deterministic.
__global__ void k_mgs_step(int64_t n, double* __restrict__ w, const double* __restrict__ vprev,
                           const double* __restrict__ hprev, const double* __restrict__ vcur,
                           double* __restrict__ part) {
  __shared__ double sh[32];
  const double hp = vprev ? *hprev : 0.0;
  double loc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double wk = w[k];
    if (vprev) {
      wk = __fma_rn(-hp, vprev[k], wk);
      w[k] = wk;
    }
    loc = __fma_rn(wk, vcur ? vcur[k] : wk, loc);
  }
  const double t = block_sum(loc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// h[i] = sum over CTAs of part[i * G + c], fixed order.
__global__ void k_reduce_parts(int nv, int G, const double* __restrict__ part, double* __restrict__ h) {
  const int i = blockIdx.x;
  if (i >= nv) return;
  double t = 0.0;
  for (int c = threadIdx.x; c < G; c += 32) t += part[(int64_t)i * G + c];
  t = warp_sum(t);
  if (threadIdx.x == 0) h[i] = t;
}

// w -= sum_i h[i] V_i  (h on the device)
__global__ void k_sub_multi(int64_t n, int nv, const double* __restrict__ V, int64_t ldv,
                            const double* __restrict__ h, double* __restrict__ w) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[k];
    for (int i = 0; i < nv; ++i) acc = __fma_rn(-h[i], V[i * ldv + k], acc);
    w[k] = acc;
  }
}

// x += sum_i y[i] Z_i  (y on the device)
__global__ void k_add_multi(int64_t n, int nv, const double* __restrict__ Z, int64_t ldz,
                            const double* __restrict__ y, double* __restrict__ x) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double acc = x[k];
    for (int i = 0; i < nv; ++i) acc = __fma_rn(y[i], Z[i * ldz + k], acc);
    x[k] = acc;
  }
}

__global__ void k_scale_to(int64_t n, const double* __restrict__ s, int invert, const double* __restrict__ a,
                           double* __restrict__ b) {
  const double f = invert ? 1.0 / *s : *s;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i] * f;
}

}  // namespace

// ============================================================== launchers

cudaError_t schur_init(int64_t nb, int64_t b0, const int64_t* prp, const int32_t* pci, const double* pv, double* SB,
                       cudaStream_t st) {
  SDSL_CUDA_TRY(cudaMemsetAsync(SB, 0, sizeof(double) * (size_t)(nb * nb), st));
  if (nb == 0) return cudaSuccess;
  k_schur_init<<<grid_for(nb, 128), 128, 0, st>>>(nb, b0, prp, pci, pv, SB); count_launch();
  return cudaGetLastError();
}

int64_t schur_tiles(int64_t nb) { return (nb + kR - 1) / kR; }

cudaError_t schur_wave(int njobs, const SchurJob* jobs, int64_t b0, int64_t nb, const int64_t* prp,
                       const int32_t* pci, const double* pv, const double* F, const double* dinv,
                       const int64_t* pdiag, const int32_t* lev_ptr_lo, const int32_t* lev_rows_lo,
                       const int32_t* lev_ptr_up, const int32_t* lev_rows_up, double* X, double* Cpart, double* SB,
                       cudaStream_t st) {
  if (njobs == 0 || nb == 0) return cudaSuccess;
  const dim3 grid((unsigned)schur_tiles(nb), (unsigned)njobs);
  k_schur_wave<<<grid, 256, 0, st>>>(jobs, b0, nb, prp, pci, pv, F, dinv, pdiag, lev_ptr_lo, lev_rows_lo, lev_ptr_up,
                                     lev_rows_up, X, Cpart); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  k_schur_reduce<<<grid_for(nb * nb, 256), 256, 0, st>>>(nb, njobs, Cpart, SB); count_launch();
  return cudaGetLastError();
}

cudaError_t dense_lu_f32(int64_t n, const double* SB, float* LU, int32_t* ipiv, double* W, double* udiag,
                         int* status, int mode, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_to_f32<<<grid_for(n * n, 256), 256, 0, st>>>(n * n, SB, LU); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  if (mode != 2) return dense_lu_blocked(n, LU, ipiv, W, udiag, status, mode == 0 ? 1 : 0, st);
  for (int64_t k = 0; k < n; ++k) {
    k_lu_pivot<<<1, 1024, 0, st>>>(n, k, LU, ipiv, status); count_launch();
    SDSL_CUDA_TRY(cudaGetLastError());
    if (k + 1 < n) {
      k_lu_update<<<(unsigned)std::min<int64_t>(n - k - 1, 1024), 256, 0, st>>>(n, k, LU); count_launch();
      SDSL_CUDA_TRY(cudaGetLastError());
    }
  }
  return cudaSuccess;
}

cudaError_t dense_lu_inverse(int64_t n, const float* LU, const int32_t* ipiv, const double* udiag, float* Xinv,
                             float* work, int mode, int* status, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (mode != 2)
    return dense_inverse_blocked(n, LU, ipiv, udiag, Xinv, reinterpret_cast<int32_t*>(work), status,
                                 mode == 0 ? 1 : 0, st);
  k_lu_inverse<<<(unsigned)((n + 31) / 32), 512, 0, st>>>(n, LU, ipiv, Xinv, work); count_launch();
  return cudaGetLastError();
}

cudaError_t block_lu_solve(int64_t nblocks, const int64_t* bp, const int64_t* prp, const int32_t* pci,
                           const double* F, const double* dinv, const int64_t* pdiag, const int32_t* lev_off_lo,
                           const int32_t* lev_ptr_lo, const int32_t* lev_rows_lo, const int32_t* lev_off_up,
                           const int32_t* lev_ptr_up, const int32_t* lev_rows_up, double* y, cudaStream_t st) {
  if (nblocks == 0) return cudaSuccess;
  k_block_lu_solve<<<(unsigned)nblocks, 512, 0, st>>>(bp, prp, pci, F, dinv, pdiag, lev_off_lo, lev_ptr_lo,
                                                      lev_rows_lo, lev_off_up, lev_ptr_up, lev_rows_up, y); count_launch();
  return cudaGetLastError();
}

cudaError_t border_gather(int64_t nb, int64_t b0, const int64_t* prp, const int32_t* pci, const double* pv,
                          const double* r, const double* t, double* g, cudaStream_t st) {
  if (nb == 0) return cudaSuccess;
  k_border_gather<<<grid_for(nb, 8), 256, 0, st>>>(nb, b0, prp, pci, pv, r, t, g); count_launch();
  return cudaGetLastError();
}

cudaError_t border_scatter(int64_t b0, const int64_t* prp, const int32_t* pci, const int64_t* pdiag,
                           const double* pv, const double* r, const double* zB, double* w, cudaStream_t st) {
  if (b0 == 0) return cudaSuccess;
  k_border_scatter<<<grid_for(b0, 256), 256, 0, st>>>(b0, prp, pci, pdiag, pv, r, zB, w); count_launch();
  return cudaGetLastError();
}

cudaError_t dense_mv(int64_t n, const float* A32, const double* A64, const double* x, const double* b, double* y,
                     int residual, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (A32) {
    k_dense_mv<float><<<grid_for(n, 8), 256, 0, st>>>(n, A32, x, b, y, residual); count_launch();
  } else {
    k_dense_mv<double><<<grid_for(n, 8), 256, 0, st>>>(n, A64, x, b, y, residual); count_launch();
  }
  return cudaGetLastError();
}

cudaError_t axpy(int64_t n, double a, const double* x, double* y, cudaStream_t st) {
  k_axpy<<<grid_for(n, 256), 256, 0, st>>>(n, a, x, y); count_launch();
  return cudaGetLastError();
}

cudaError_t copy_vec(int64_t n, const double* a, double* b, cudaStream_t st) {
  k_copy_range<<<grid_for(n, 256), 256, 0, st>>>(n, a, b); count_launch();
  return cudaGetLastError();
}

int multidot_grid(int64_t n) { return (int)grid_for(n, 256, 152 * 4); }

cudaError_t multidot(int64_t n, int nv, const double* V, int64_t ldv, const double* w, double* part, double* h,
                     cudaStream_t st) {
  const int G = multidot_grid(n);
  k_multidot<<<G, 256, 0, st>>>(n, nv, V, ldv, w, part); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  k_reduce_parts<<<nv, 32, 0, st>>>(nv, G, part, h); count_launch();
  return cudaGetLastError();
}

cudaError_t mgs_step(int64_t n, double* w, const double* vprev, const double* hprev, const double* vcur, double* part,
                     double* hout, cudaStream_t st) {
  const int G = multidot_grid(n);
  k_mgs_step<<<G, 256, 0, st>>>(n, w, vprev, hprev, vcur, part); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  k_reduce_parts<<<1, 32, 0, st>>>(1, G, part, hout); count_launch();
  return cudaGetLastError();
}

cudaError_t sub_multi(int64_t n, int nv, const double* V, int64_t ldv, const double* h, double* w, cudaStream_t st) {
  k_sub_multi<<<grid_for(n, 256), 256, 0, st>>>(n, nv, V, ldv, h, w); count_launch();
  return cudaGetLastError();
}

cudaError_t add_multi(int64_t n, int nv, const double* Z, int64_t ldz, const double* y, double* x, cudaStream_t st) {
  k_add_multi<<<grid_for(n, 256), 256, 0, st>>>(n, nv, Z, ldz, y, x); count_launch();
  return cudaGetLastError();
}

cudaError_t scale_to(int64_t n, const double* s, int invert, const double* a, double* b, cudaStream_t st) {
  k_scale_to<<<grid_for(n, 256), 256, 0, st>>>(n, s, invert, a, b); count_launch();
  return cudaGetLastError();
}

}  // namespace sdsl
