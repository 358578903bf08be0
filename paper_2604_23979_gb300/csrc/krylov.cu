// krylov.cu -- kernels of the Krylov iterations (Sec. 2.2-2.3).
//
// One PCG iteration (right-preconditioned CG, Block Jacobi M) is three
// launches, captured in a CUDA graph by the host:
//   k_pcg_spmv      q = S p and p^T q                  (CSR SpMV, V lanes/row)
//   k_pcg_update    x += a p, r -= a q, ||r||^2, z = M^{-1} r per block
//                   (level-scheduled forward/backward solves, one CTA per
//                   block, y staged in shared memory), r^T z
//   k_pcg_direction p = z + b p
// Inner products are two-stage and deterministic: per-CTA partials in a fixed
// order, then the last CTA to finish (atomic ticket) sums them in a fixed
// order and writes the scalars for the next launch into PcgState.  The
// paper's MPI_Allreduce of the inner products (Sec. 2.3) becomes this
// on-device reduction; the ghost exchange disappears (x is resident).
#include "common.cuh"
#include "kernels.cuh"

namespace sdsl {

namespace {

constexpr int kThreads = 256;

// Deterministic sum of a[0, n) by one warp (lane-strided, then butterfly).
__device__ __forceinline__ double warp_fixed_sum(const double* a, int n) {
  double t = 0.0;
  for (int i = lane_id(); i < n; i += 32) t += a[i];
  return warp_sum(t);
}

// Returns true in every thread of the last CTA to arrive.
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
  __shared__ int amlast;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) amlast = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (amlast) __threadfence();
  return amlast;
}

// Row i of A times x by the V lanes of a group.  Every lane of the warp must
// call it (the group shuffle uses the full mask); lanes of a group without a
// row pass valid = false.
template <int V>
__device__ __forceinline__ double row_dot(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                          const double* __restrict__ v, const double* __restrict__ x, int64_t i,
                                          int sub, bool valid) {
  double acc = 0.0;
  if (valid) {
    const int64_t s = rp[i], e = rp[i + 1];
    for (int64_t t = s + sub; t < e; t += V) acc = __fma_rn(v[t], __ldg(x + ci[t]), acc);
  }
  return group_sum<V>(acc);
}

// Row range of CTA c: rows split evenly (deterministic for a fixed grid).
__device__ __forceinline__ void cta_rows(int64_t n, int64_t& r0, int64_t& r1) {
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  r0 = (int64_t)blockIdx.x * per;
  r1 = min(n, r0 + per);
}

template <int V>
__global__ void __launch_bounds__(kThreads) k_spmv(int64_t n, const int64_t* __restrict__ rp,
                                                   const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                   const double* __restrict__ x, double* __restrict__ y) {
  int64_t r0, r1;
  cta_rows(n, r0, r1);
  const int g = threadIdx.x / V, sub = threadIdx.x % V, ng = kThreads / V;
  for (int64_t base = r0; base < r1; base += ng) {
    const int64_t i = base + g;
    const bool valid = i < r1;
    const double acc = row_dot<V>(rp, ci, v, x, i, sub, valid);
    if (valid && sub == 0) y[i] = acc;
  }
}

template <int V>
__global__ void __launch_bounds__(kThreads) k_pcg_spmv(int64_t n, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                       const double* __restrict__ p, double* __restrict__ q,
                                                       double* __restrict__ part, PcgState* __restrict__ s) {
  if (s->done) return;
  __shared__ double sh[kThreads / 32];
  int64_t r0, r1;
  cta_rows(n, r0, r1);
  const int g = threadIdx.x / V, sub = threadIdx.x % V, ng = kThreads / V;
  double loc = 0.0;
  for (int64_t base = r0; base < r1; base += ng) {
    const int64_t i = base + g;
    const bool valid = i < r1;
    const double acc = row_dot<V>(rp, ci, v, p, i, sub, valid);
    if (valid && sub == 0) {
      q[i] = acc;
      loc = __fma_rn(p[i], acc, loc);
    }
  }
  const double tot = block_sum(loc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
  if (last_block(&s->ticket[0])) {
    if (threadIdx.x < 32) {
      const double pq = warp_fixed_sum(part, gridDim.x);
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

// t = b - A x, ||t||^2 -> s->tr; optionally r = t.
template <int V>
__global__ void __launch_bounds__(kThreads) k_residual(int64_t n, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                       const double* __restrict__ b, const double* __restrict__ x,
                                                       double* __restrict__ r, double* __restrict__ part,
                                                       PcgState* __restrict__ s, int write_r) {
  __shared__ double sh[kThreads / 32];
  int64_t r0, r1;
  cta_rows(n, r0, r1);
  const int g = threadIdx.x / V, sub = threadIdx.x % V, ng = kThreads / V;
  double loc = 0.0;
  for (int64_t base = r0; base < r1; base += ng) {
    const int64_t i = base + g;
    const bool valid = i < r1;
    const double ax = row_dot<V>(rp, ci, v, x, i, sub, valid);
    if (valid && sub == 0) {
      const double t = b[i] - ax;
      if (write_r) r[i] = t;
      loc = __fma_rn(t, t, loc);
    }
  }
  const double tot = block_sum(loc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
  if (last_block(&s->ticket[1])) {
    if (threadIdx.x < 32) {
      const double tr = warp_fixed_sum(part, gridDim.x);
      if (threadIdx.x == 0) {
        s->tr = tr;
        s->ticket[1] = 0;
      }
    }
  }
}

__global__ void k_norm2(int64_t n, const double* __restrict__ a, double* __restrict__ part, double* __restrict__ out,
                        unsigned int* ticket) {
  __shared__ double sh[kThreads / 32];
  double loc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    loc = __fma_rn(a[i], a[i], loc);
  const double tot = block_sum(loc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
  if (last_block(ticket)) {
    if (threadIdx.x < 32) {
      const double t = warp_fixed_sum(part, gridDim.x);
      if (threadIdx.x == 0) {
        *out = t;
        *ticket = 0;
      }
    }
  }
}

// Level-scheduled block triangular solves on y (staged in `ybuf`, indexed by
// row - s0).  Forward: y_i = (y_i - sum_{j<i} L_ij y_j) * dinv_i (unit L: no
// scaling); backward: y_i = (y_i - sum_{j>i} U_ij y_j) * dinv_i.
template <typename T, int V>
__device__ __forceinline__ void block_solve(const TriSolve& M, const T* __restrict__ F, const T* __restrict__ dinv,
                                           int b, int64_t s0, T* ybuf) {
  const int g = threadIdx.x / V, sub = threadIdx.x % V, ng = blockDim.x / V;
  const int64_t* __restrict__ prp = M.prp;
  const int32_t* __restrict__ pci = M.pci;
  const int64_t* __restrict__ pdiag = M.pdiag;
  for (int32_t L = M.lev_off_lo[b]; L < M.lev_off_lo[b + 1]; ++L) {
    const int32_t q0 = M.lev_ptr_lo[L], q1 = M.lev_ptr_lo[L + 1];
    for (int32_t base = q0; base < q1; base += ng) {  // uniform trip count: shuffles need every lane
      const int32_t idx = base + g;
      const bool valid = idx < q1;
      const int64_t i = valid ? M.lev_rows_lo[idx] : 0;
      T acc = T(0);
      if (valid)
        for (int64_t t = prp[i] + sub; t < pdiag[i]; t += V) acc += F[t] * ybuf[pci[t] - s0];
      acc = group_sum<V>(acc);
      if (valid && sub == 0) {
        const T yi = ybuf[i - s0] - acc;
        ybuf[i - s0] = M.unit_lower ? yi : yi * dinv[i];
      }
    }
    __syncthreads();
  }
  for (int32_t L = M.lev_off_up[b]; L < M.lev_off_up[b + 1]; ++L) {
    const int32_t q0 = M.lev_ptr_up[L], q1 = M.lev_ptr_up[L + 1];
    for (int32_t base = q0; base < q1; base += ng) {
      const int32_t idx = base + g;
      const bool valid = idx < q1;
      const int64_t i = valid ? M.lev_rows_up[idx] : 0;
      T acc = T(0);
      if (valid) {
        const int64_t e = prp[i + 1];
        for (int64_t t = pdiag[i] + 1 + sub; t < e; t += V) acc += F[t] * ybuf[pci[t] - s0];
      }
      acc = group_sum<V>(acc);
      if (valid && sub == 0) ybuf[i - s0] = (ybuf[i - s0] - acc) * dinv[i];
    }
    __syncthreads();
  }
}

// mode 0: PCG update + preconditioner; mode 1: z = M^{-1} r only, then
// rho = r^T z and p = z (start / restart of PCG); mode 2: z = M^{-1} r only.
template <typename T, int V, bool kSmem>
__global__ void __launch_bounds__(kThreads) k_pcg_update(TriSolve M, const double* __restrict__ p,
                                                         const double* __restrict__ q, double* __restrict__ x,
                                                         double* __restrict__ r, double* __restrict__ z,
                                                         double* __restrict__ pp, double* __restrict__ part_rr,
                                                         double* __restrict__ part_rz, PcgState* __restrict__ s,
                                                         int mode) {
  if (mode == 0 && s->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[kThreads / 32];
  const int b = blockIdx.x;
  const int64_t s0 = M.bp[b], e0 = M.bp[b + 1];
  T* ybuf;
  if (kSmem) {
    ybuf = reinterpret_cast<T*>(smem_raw);
  } else {
    ybuf = (sizeof(T) == 4) ? reinterpret_cast<T*>(M.yscratch + s0) : reinterpret_cast<T*>(M.yscratch64 + s0);
  }
  const T* F = (sizeof(T) == 4) ? reinterpret_cast<const T*>(M.Ff) : reinterpret_cast<const T*>(M.F);
  const T* dinv = (sizeof(T) == 4) ? reinterpret_cast<const T*>(M.dinvf) : reinterpret_cast<const T*>(M.dinv);
  double rr = 0.0;
  if (mode == 0) {
    const double a = s->alpha;
    for (int64_t i = s0 + threadIdx.x; i < e0; i += blockDim.x) {
      const double ri = __fma_rn(-a, q[i], r[i]);
      x[i] = __fma_rn(a, p[i], x[i]);
      r[i] = ri;
      rr = __fma_rn(ri, ri, rr);
      ybuf[i - s0] = (T)ri;
    }
  } else {
    for (int64_t i = s0 + threadIdx.x; i < e0; i += blockDim.x) {
      const double ri = r[i];
      rr = __fma_rn(ri, ri, rr);
      ybuf[i - s0] = (T)ri;
    }
  }
  const double rrb = block_sum(rr, sh);
  __syncthreads();
  block_solve<T, V>(M, F, dinv, b, s0, ybuf);
  double rz = 0.0;
  for (int64_t i = s0 + threadIdx.x; i < e0; i += blockDim.x) {
    const double zi = (double)ybuf[i - s0];
    z[i] = zi;
    if (mode == 1) pp[i] = zi;
    rz = __fma_rn(r[i], zi, rz);
  }
  const double rzb = block_sum(rz, sh);
  if (threadIdx.x == 0) {
    part_rr[b] = rrb;
    part_rz[b] = rzb;
  }
  if (mode == 2) return;
  if (last_block(&s->ticket[2])) {
    if (threadIdx.x < 32) {
      const double rrt = warp_fixed_sum(part_rr, gridDim.x);
      const double rzt = warp_fixed_sum(part_rz, gridDim.x);
      if (threadIdx.x == 0) {
        s->rr = rrt;
        s->rz_new = rzt;
        if (mode == 0) {
          if (rrt <= s->tol2) s->done = 1;
          else if (s->iters >= s->maxit) s->done = 2;
          else if (!isfinite(rzt) || !isfinite(rrt)) s->done = 3;
          s->beta = rzt / s->rho;
          s->rho = rzt;
        } else {
          s->rho = rzt;
        }
        s->ticket[2] = 0;
      }
    }
  }
}

__global__ void k_pcg_direction(int64_t n, const double* __restrict__ z, double* __restrict__ p,
                                const PcgState* __restrict__ s) {
  if (s->done) return;
  const double beta = s->beta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = __fma_rn(beta, p[i], z[i]);
}

__global__ void k_init_state(PcgState* s, double tol2, long long maxit) {
  PcgState t = {};
  t.tol2 = tol2;
  t.maxit = maxit;
  *s = t;
}

template <typename F>
cudaError_t by_lanes(int lanes, F&& f) {
  switch (lanes) {
    case 2: return f(std::integral_constant<int, 2>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    default: return f(std::integral_constant<int, 32>{});
  }
}

inline unsigned grid_for(int64_t work, int per_block, int cap = 152 * 16) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (unsigned)g;
}

template <typename T, int V>
cudaError_t launch_update(const TriSolve& M, const double* p, const double* q, double* x, double* r, double* z,
                          double* pp, double* part_rr, double* part_rz, PcgState* s, int mode, cudaStream_t st) {
  const size_t need = (size_t)M.max_block * sizeof(T);
  if (need <= (size_t)200 * 1024) {
    auto kern = k_pcg_update<T, V, true>;
    SDSL_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
    kern<<<(unsigned)M.nblocks, kThreads, need, st>>>(M, p, q, x, r, z, pp, part_rr, part_rz, s, mode);
  } else {
    k_pcg_update<T, V, false><<<(unsigned)M.nblocks, kThreads, 0, st>>>(M, p, q, x, r, z, pp, part_rr, part_rz, s,
                                                                        mode);
  }
  return cudaGetLastError();
}

cudaError_t update_any(const TriSolve& M, const double* p, const double* q, double* x, double* r, double* z,
                       double* pp, double* part_rr, double* part_rz, PcgState* s, int mode, cudaStream_t st) {
  return by_lanes(M.lanes, [&](auto V) -> cudaError_t {
    if (M.prec == 32) return launch_update<float, decltype(V)::value>(M, p, q, x, r, z, pp, part_rr, part_rz, s, mode, st);
    return launch_update<double, decltype(V)::value>(M, p, q, x, r, z, pp, part_rr, part_rz, s, mode, st);
  });
}

}  // namespace

cudaError_t spmv(const SpmvPlan& A, const double* x, double* y, cudaStream_t st) {
  return by_lanes(A.lanes, [&](auto V) -> cudaError_t {
    k_spmv<decltype(V)::value><<<A.grid, kThreads, 0, st>>>(A.n, A.rp, A.ci, A.v, x, y);
    return cudaGetLastError();
  });
}

cudaError_t pcg_spmv(const SpmvPlan& A, const double* p, double* q, double* part, PcgState* s, cudaStream_t st) {
  return by_lanes(A.lanes, [&](auto V) -> cudaError_t {
    k_pcg_spmv<decltype(V)::value><<<A.grid, kThreads, 0, st>>>(A.n, A.rp, A.ci, A.v, p, q, part, s);
    return cudaGetLastError();
  });
}

cudaError_t pcg_update_precond(const TriSolve& M, const double* p, const double* q, double* x, double* r, double* z,
                               double* part_rr, double* part_rz, PcgState* s, cudaStream_t st) {
  return update_any(M, p, q, x, r, z, nullptr, part_rr, part_rz, s, 0, st);
}

cudaError_t precond_apply(const TriSolve& M, const double* r, double* z, double* p_out, double* part_rr,
                          double* part_rz, PcgState* s, int mode, cudaStream_t st) {
  return update_any(M, nullptr, nullptr, nullptr, const_cast<double*>(r), z, p_out, part_rr, part_rz, s, mode, st);
}

cudaError_t pcg_direction(int64_t n, const double* z, double* p, PcgState* s, cudaStream_t st) {
  k_pcg_direction<<<grid_for(n, kThreads), kThreads, 0, st>>>(n, z, p, s);
  return cudaGetLastError();
}

cudaError_t true_residual(const SpmvPlan& A, const double* b, const double* x, double* r, double* part,
                          PcgState* s, int write_r, cudaStream_t st) {
  return by_lanes(A.lanes, [&](auto V) -> cudaError_t {
    k_residual<decltype(V)::value><<<A.grid, kThreads, 0, st>>>(A.n, A.rp, A.ci, A.v, b, x, r, part, s, write_r);
    return cudaGetLastError();
  });
}

cudaError_t norm2_sq(int64_t n, const double* a, double* part, double* out, unsigned int* ticket, cudaStream_t st) {
  const unsigned g = grid_for(n, kThreads, 152 * 4);
  k_norm2<<<g, kThreads, 0, st>>>(n, a, part, out, ticket);
  return cudaGetLastError();
}

cudaError_t pcg_init_state(PcgState* s, double tol2, long long maxit, cudaStream_t st) {
  k_init_state<<<1, 1, 0, st>>>(s, tol2, maxit);
  return cudaGetLastError();
}

}  // namespace sdsl
