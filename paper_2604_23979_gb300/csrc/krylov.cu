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
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"
#include "pcg_common.cuh"

namespace sdsl {

namespace {

constexpr int kThreads = 256;


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
    int64_t t = s + sub;
    // Four independent column/value loads in flight per lane before the
    // gathers (memory-level parallelism) and four independent accumulators
    // (no FMA latency chain).  S is streamed (evict-first); x is gathered
    // through the read-only path and stays in L2.  On GB300 the FP64 pipe is
    // a co-bound of this kernel, so few lanes per row (long per-lane runs,
    // one shuffle reduction per row) keep FP64 instructions close to one
    // per nonzero.
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (; t + 3 * V < e; t += 4 * V) {
      const int32_t c0 = __ldcs(ci + t), c1 = __ldcs(ci + t + V), c2 = __ldcs(ci + t + 2 * V),
                    c3 = __ldcs(ci + t + 3 * V);
      const double v0 = __ldcs(v + t), v1 = __ldcs(v + t + V), v2 = __ldcs(v + t + 2 * V), v3 = __ldcs(v + t + 3 * V);
      const double x0 = __ldg(x + c0), x1 = __ldg(x + c1), x2 = __ldg(x + c2), x3 = __ldg(x + c3);
      a0 = __fma_rn(v0, x0, a0);
      a1 = __fma_rn(v1, x1, a1);
      a2 = __fma_rn(v2, x2, a2);
      a3 = __fma_rn(v3, x3, a3);
    }
    for (; t < e; t += V) a0 = __fma_rn(__ldcs(v + t), __ldg(x + __ldcs(ci + t)), a0);
    acc = (a0 + a1) + (a2 + a3);
  }
  return group_sum<V>(acc);
}

// Long rows (more than thr entries): their product values were computed by
// k_long_dot into ax[k] (k = position of the row in the ascending list).
struct LongRows {
  int thr;
  int64_t n;
  const int32_t* rows;
  const double* ax;
};

__device__ __forceinline__ double long_value(const LongRows& L, int64_t i) {
  int64_t lo = 0, hi = L.n - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (L.rows[mid] < i) lo = mid + 1; else hi = mid;
  }
  return L.ax[lo];
}

// Row i of A times x (every lane of the warp calls it), long rows excepted.
template <int V>
__device__ __forceinline__ double row_value(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                            const double* __restrict__ v, const double* __restrict__ x, int64_t i,
                                            int sub, bool valid, const LongRows& L) {
  const bool lng = valid && L.thr > 0 && rp[i + 1] - rp[i] > L.thr;
  const double acc = row_dot<V>(rp, ci, v, x, i, sub, valid && !lng);
  return lng ? long_value(L, i) : acc;
}

// One CTA per long row: a[k] = row long_rows[k] of A times x, summed by the
// whole CTA in a fixed order (deterministic).
__global__ void __launch_bounds__(kThreads) k_long_dot(int64_t n_long, const int32_t* __restrict__ rows,
                                                       const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                       const double* __restrict__ x, double* __restrict__ ax,
                                                       const PcgState* __restrict__ s) {
  if (s && s->done) return;
  __shared__ double sh[kThreads / 32];
  for (int64_t k = blockIdx.x; k < n_long; k += gridDim.x) {
    const int64_t i = rows[k];
    double a0 = 0.0, a1 = 0.0;
    const int64_t e = rp[i + 1];
    int64_t t = rp[i] + threadIdx.x;
    for (; t + kThreads < e; t += 2 * kThreads) {
      a0 = __fma_rn(__ldcs(v + t), __ldg(x + __ldcs(ci + t)), a0);
      a1 = __fma_rn(__ldcs(v + t + kThreads), __ldg(x + __ldcs(ci + t + kThreads)), a1);
    }
    if (t < e) a0 = __fma_rn(__ldcs(v + t), __ldg(x + __ldcs(ci + t)), a0);
    const double tot = block_sum(a0 + a1, sh);
    if (threadIdx.x == 0) ax[k] = tot;
    __syncthreads();
  }
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
                                                   const double* __restrict__ x, double* __restrict__ y,
                                                   LongRows L) {
  int64_t r0, r1;
  cta_rows(n, r0, r1);
  const int g = threadIdx.x / V, sub = threadIdx.x % V, ng = kThreads / V;
  for (int64_t base = r0; base < r1; base += ng) {
    const int64_t i = base + g;
    const bool valid = i < r1;
    const double acc = row_value<V>(rp, ci, v, x, i, sub, valid, L);
    if (valid && sub == 0) y[i] = acc;
  }
}

template <int V>
__global__ void __launch_bounds__(kThreads) k_pcg_spmv(int64_t n, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                       const double* __restrict__ p, double* __restrict__ q,
                                                       double* __restrict__ part, PcgState* __restrict__ s,
                                                       LongRows L) {
  if (s->done) return;
  __shared__ double sh[kThreads / 32];
  int64_t r0, r1;
  cta_rows(n, r0, r1);
  const int g = threadIdx.x / V, sub = threadIdx.x % V, ng = kThreads / V;
  double loc = 0.0;
  for (int64_t base = r0; base < r1; base += ng) {
    const int64_t i = base + g;
    const bool valid = i < r1;
    const double acc = row_value<V>(rp, ci, v, p, i, sub, valid, L);
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

// Factored normal-equation product, first half: u = theta o (A^T p).
template <int V>
__global__ void __launch_bounds__(kThreads) k_at_theta(int64_t n, const int64_t* __restrict__ at_rp,
                                                       const int32_t* __restrict__ at_ci,
                                                       const double* __restrict__ at_v,
                                                       const double* __restrict__ theta,
                                                       const double* __restrict__ p, double* __restrict__ u,
                                                       const PcgState* __restrict__ s) {
  if (s && s->done) return;
  int64_t r0, r1;
  cta_rows(n, r0, r1);
  const int g = threadIdx.x / V, sub = threadIdx.x % V, ng = kThreads / V;
  for (int64_t base = r0; base < r1; base += ng) {
    const int64_t k = base + g;
    const bool valid = k < r1;
    const double acc = row_dot<V>(at_rp, at_ci, at_v, p, k, sub, valid);
    if (valid && sub == 0) u[k] = theta[k] * acc;
  }
}

// Second half: q = A u + rho p, partial p^T q; last CTA: alpha, iters.
template <int V>
__global__ void __launch_bounds__(kThreads) k_a_u_dot(int64_t m, const int64_t* __restrict__ a_rp,
                                                      const int32_t* __restrict__ a_ci,
                                                      const double* __restrict__ a_v, const double* __restrict__ u,
                                                      double rho, const double* __restrict__ p,
                                                      double* __restrict__ q, double* __restrict__ part,
                                                      PcgState* __restrict__ s, int pcg) {
  if (pcg && s->done) return;
  __shared__ double sh[kThreads / 32];
  int64_t r0, r1;
  cta_rows(m, r0, r1);
  const int g = threadIdx.x / V, sub = threadIdx.x % V, ng = kThreads / V;
  double loc = 0.0;
  for (int64_t base = r0; base < r1; base += ng) {
    const int64_t i = base + g;
    const bool valid = i < r1;
    const double acc = row_dot<V>(a_rp, a_ci, a_v, u, i, sub, valid);
    if (valid && sub == 0) {
      const double qi = __fma_rn(rho, p[i], acc);
      q[i] = qi;
      loc = __fma_rn(p[i], qi, loc);
    }
  }
  if (pcg != 1) return;
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
                                                       PcgState* __restrict__ s, int write_r, LongRows L) {
  __shared__ double sh[kThreads / 32];
  int64_t r0, r1;
  cta_rows(n, r0, r1);
  const int g = threadIdx.x / V, sub = threadIdx.x % V, ng = kThreads / V;
  double loc = 0.0;
  for (int64_t base = r0; base < r1; base += ng) {
    const int64_t i = base + g;
    const bool valid = i < r1;
    const double ax = row_value<V>(rp, ci, v, x, i, sub, valid, L);
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


// Level-synchronous variant (any block size): y staged in shared memory if
// the largest block fits, else in a global scratch vector.
// mode 0: PCG update + preconditioner; mode 1: z = M^{-1} r only, then
// rho = r^T z and p = z (start / restart of PCG); mode 2: z = M^{-1} r only.
template <typename T, int V, bool kSmem>
__global__ void __launch_bounds__(kThreads) k_pcg_update(TriSolve M, const double* __restrict__ p,
                                                         const double* __restrict__ q, double* __restrict__ x,
                                                         double* __restrict__ r, double* __restrict__ z,
                                                         double* __restrict__ pp, double* __restrict__ part,
                                                         PcgState* __restrict__ s, int mode) {
  if ((mode == 0 || mode == 3) && s->done) return;
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
  double rz = 0.0, zq = 0.0;
  for (int64_t i = s0 + threadIdx.x; i < e0; i += blockDim.x) {
    const double zi = (double)ybuf[i - s0];
    z[i] = zi;
    if (mode == 1) pp[i] = zi;
    rz = __fma_rn(r[i], zi, rz);
    if (mode == 0) zq = __fma_rn(zi, q[i], zq);
  }
  const double rzb = block_sum(rz, sh);
  const double zqb = block_sum(zq, sh);
  update_epilogue(M, rrb, rzb, zqb, part, s, mode, false, (int)blockIdx.x);
}

// Sum over the V lanes of this thread's group only, so that the groups of a
// warp stay independent while they wait on flags.
template <int V, typename T>
__device__ __forceinline__ T group_sum_own(T v) {
  if (V == 32) return warp_sum(v);
  const unsigned mask = ((1u << V) - 1u) << (lane_id() & ~(unsigned)(V - 1));
#pragma unroll
  for (int o = V / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

constexpr int kPre = 4;              // entries per lane prefetched one position ahead

template <typename TS, typename TC>
struct RowPre {  // registers of one prefetched position
  int i;
  int64_t a, e;
  TC d;
  int j[kPre];
  TC v[kPre];
};

// Stage 1 of the prefetch (two tiles ahead): row metadata only.
template <typename TS, typename TC>
__device__ __forceinline__ void load_meta(RowPre<TS, TC>& R, const int64_t* __restrict__ off,
                                          const TS* __restrict__ pdinv, const int32_t* __restrict__ prow, int64_t q) {
  R.i = prow[q];
  R.a = off[q];
  R.e = off[q + 1];
  R.d = (TC)pdinv[q];
}

// Stage 2 (one tile ahead): the entries, addressed by metadata that arrived
// one step earlier -- so no load waits on a load issued in the same step
// (instruction issue is in order: a dependent load would stall the warp).
template <typename TS, typename TC, int V>
__device__ __forceinline__ void load_entries(RowPre<TS, TC>& R, const int32_t* __restrict__ col,
                                             const TS* __restrict__ val, int sub) {
#pragma unroll
  for (int k = 0; k < kPre; ++k) {
    const int64_t t = R.a + sub + (int64_t)k * V;
    if (t < R.e) {
      R.j[k] = col[t];
      R.v[k] = (TC)val[t];
    } else {
      R.j[k] = -1;
      R.v[k] = TC(0);
    }
  }
}

template <typename TS, typename TC, int V>
__device__ __forceinline__ void load_pos(RowPre<TS, TC>& R, const int64_t* __restrict__ off,
                                         const int32_t* __restrict__ col, const TS* __restrict__ val,
                                         const TS* __restrict__ pdinv, const int32_t* __restrict__ prow, int64_t q,
                                         int sub) {
  R.i = prow[q];
  R.a = off[q];
  R.e = off[q + 1];
  R.d = (TC)pdinv[q];
#pragma unroll
  for (int k = 0; k < kPre; ++k) {
    const int64_t t = R.a + sub + (int64_t)k * V;
    if (t < R.e) {
      R.j[k] = col[t];
      R.v[k] = (TC)val[t];
    } else {
      R.j[k] = -1;
      R.v[k] = TC(0);
    }
  }
}


// Read y[j] once it has been solved (bounded wait).
// The wait backs off with a short sleep between polls: dozens of warps
// polling shared memory back to back saturate the shared-memory pipe and
// delay the very loads and stores that resolve the waits.
template <typename TC>
__device__ __forceinline__ TC await(volatile TC* y, int j, int* timeout) {
  TC v = y[j];
  int spins = 0;
  while (is_sentinel(v)) {
    if (++spins > kSpinLimit / 8) { *timeout = 1; return TC(0); }
    __nanosleep(kBackoffNs);
    v = y[j];
  }
  return v;
}

// One flag-free sweep over a block.  The block's rows are listed in level
// order, each level padded to a whole number of warp tiles of RW = 32/V rows
// (padding positions have row -1), so the rows that one warp solves together
// belong to one level and never depend on each other.  Warp w takes tiles
// w, w+W, ... in increasing order; every lane reads the entries of its row
// (prefetched one tile ahead), waits for each column's value to be solved
// and accumulates; the group's first lane writes the row's value.  Every
// dependency of a tile lies in a lower level, i.e. in an earlier tile, so
// the earliest unfinished tile can always proceed and the sweep cannot
// deadlock; every wait is bounded anyway.
//   in:  right-hand side of the sweep (indexed by block row)
//   out: solved values, all equal to the sentinel on entry
template <typename TS, typename TC, int V>
__device__ void sweep(const int64_t* __restrict__ off, const int32_t* __restrict__ col, const TS* __restrict__ val,
                      const TS* __restrict__ pdinv, const int32_t* __restrict__ prow, int64_t q0, int64_t npos,
                      volatile TC* in, volatile TC* out, bool unit, int* timeout) {
  constexpr int RW = 32 / V;
  const int lane = lane_id(), w = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int slot = lane / V, sub = lane % V;
  const int64_t ntiles = npos / RW;
  if (w >= ntiles) return;
  RowPre<TS, TC> nx, nn;  // next tile (entries loaded), tile after next (metadata loaded)
  load_pos<TS, TC, V>(nx, off, col, val, pdinv, prow, q0 + (int64_t)w * RW + slot, sub);
  if (w + W < ntiles) load_meta<TS, TC>(nn, off, pdinv, prow, q0 + (int64_t)(w + W) * RW + slot);
  for (int64_t t = w; t < ntiles; t += W) {
    const RowPre<TS, TC> cur = nx;
    if (t + W < ntiles) {
      nx = nn;
      load_entries<TS, TC, V>(nx, col, val, sub);
    }
    if (t + 2 * W < ntiles) load_meta<TS, TC>(nn, off, pdinv, prow, q0 + (t + 2 * W) * RW + slot);
    TC acc = TC(0);
#pragma unroll
    for (int k = 0; k < kPre; ++k)
      if (cur.j[k] >= 0) acc = fma(cur.v[k], await(out, cur.j[k], timeout), acc);
    for (int64_t tt = cur.a + (int64_t)kPre * V + sub; tt < cur.e; tt += V)  // rows longer than kPre*V
      acc = fma((TC)val[tt], await(out, col[tt], timeout), acc);
    acc = group_sum<V>(acc);
    if (sub == 0 && cur.i >= 0) {
      TC yi = in[cur.i] - acc;
      if (!unit) yi *= cur.d;
      out[cur.i] = yi;
    }
  }
}

// Flag-free variant: the forward input / backward output (yb) and the
// forward output (yf) of the block in shared memory (compute precision TC);
// packed level-ordered factors (storage TS).
template <typename TS, typename TC, int V>
__global__ void __launch_bounds__(1024) k_pcg_update_sf(TriSolve M, const double* __restrict__ p,
                                                        const double* __restrict__ q, double* __restrict__ x,
                                                        double* __restrict__ r, double* __restrict__ z,
                                                        double* __restrict__ pp, double* __restrict__ part,
                                                        PcgState* __restrict__ s, int mode) {
  if ((mode == 0 || mode == 3) && s->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sh[32];
  __shared__ int timeout;
  const int b = blockIdx.x;
  const int64_t s0 = M.bp[b], e0 = M.bp[b + 1];
  volatile TC* yb = reinterpret_cast<volatile TC*>(smem_raw);
  volatile TC* yf = reinterpret_cast<volatile TC*>(smem_raw + (((size_t)M.max_block * sizeof(TC) + 15) & ~(size_t)15));
  if (threadIdx.x == 0) timeout = 0;
  const TC S = sentinel(TC(0));
  double rr = 0.0;
  if (mode == 0) {
    const double a = s->alpha;
    for (int64_t i = s0 + threadIdx.x; i < e0; i += blockDim.x) {
      const double ri = __fma_rn(-a, q[i], r[i]);
      x[i] = __fma_rn(a, p[i], x[i]);
      r[i] = ri;
      rr = __fma_rn(ri, ri, rr);
      yb[i - s0] = (TC)ri;
      yf[i - s0] = S;
    }
  } else {
    for (int64_t i = s0 + threadIdx.x; i < e0; i += blockDim.x) {
      const double ri = r[i];
      rr = __fma_rn(ri, ri, rr);
      yb[i - s0] = (TC)ri;
      yf[i - s0] = S;
    }
  }
  const double rrb = block_sum(rr, sh);
  __syncthreads();
  sweep<TS, TC, V>(M.fwd_off, M.fwd_col, static_cast<const TS*>(M.fwd_val), static_cast<const TS*>(M.fwd_dinv),
                   M.fwd_row, M.fwd_pos[b], M.fwd_pos[b + 1] - M.fwd_pos[b], yb, yf, M.unit_lower != 0, &timeout);
  __syncthreads();
  for (int64_t i = threadIdx.x; i < e0 - s0; i += blockDim.x) yb[i] = S;
  __syncthreads();
  sweep<TS, TC, V>(M.bwd_off, M.bwd_col, static_cast<const TS*>(M.bwd_val), static_cast<const TS*>(M.bwd_dinv),
                   M.bwd_row, M.bwd_pos[b], M.bwd_pos[b + 1] - M.bwd_pos[b], yf, yb, false, &timeout);
  __syncthreads();
  double rz = 0.0, zq = 0.0;
  for (int64_t i = s0 + threadIdx.x; i < e0; i += blockDim.x) {
    const double zi = (double)yb[i - s0];
    z[i] = zi;
    if (mode == 1) pp[i] = zi;
    rz = __fma_rn(r[i], zi, rz);
    if (mode == 0) zq = __fma_rn(zi, q[i], zq);
  }
  const double rzb = block_sum(rz, sh);
  const double zqb = block_sum(zq, sh);
  update_epilogue(M, rrb, rzb, zqb, part, s, mode, timeout != 0, (int)blockIdx.x);
}

__device__ __forceinline__ void direction_body(int64_t n, const double* __restrict__ z, double* __restrict__ p,
                                               double beta, int vb, int vg) {
  for (int64_t i = (int64_t)vb * blockDim.x + threadIdx.x; i < n; i += (int64_t)vg * blockDim.x)
    p[i] = __fma_rn(beta, p[i], z[i]);
}

__global__ void k_pcg_direction(int64_t n, const double* __restrict__ z, double* __restrict__ p,
                                const PcgState* __restrict__ s) {
  if (s->done) return;
  direction_body(n, z, p, s->beta, (int)blockIdx.x, (int)gridDim.x);
}

// p = z + beta p for several requests in one persistent launch (items of
// each request's own grid).
__global__ void k_batch_direction(const BatchReq* __restrict__ reqs, const BatchItem* __restrict__ items,
                                  int nitems) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BatchItem I = items[it];
    const BatchReq& R = reqs[I.req];
    if (R.s->done) continue;  // no barrier in this body: per-thread decisions are safe
    direction_body(R.n, R.z, R.p, R.s->beta, I.vb, R.g_dir);
  }
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
    case 1: return f(std::integral_constant<int, 1>{});
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
                          double* pp, double* part, PcgState* s, int mode, cudaStream_t st) {
  const size_t need = (size_t)M.max_block * sizeof(T);
  if (need <= (size_t)200 * 1024) {
    auto kern = k_pcg_update<T, V, true>;
    SDSL_CUDA_TRY((allow_max_dynamic_smem<k_pcg_update<T, V, true>>()));
    kern<<<(unsigned)M.nblocks, kThreads, need, st>>>(M, p, q, x, r, z, pp, part, s, mode); count_launch();
  } else {
    k_pcg_update<T, V, false><<<(unsigned)M.nblocks, kThreads, 0, st>>>(M, p, q, x, r, z, pp, part, s, mode); count_launch();
  }
  return cudaGetLastError();
}

template <typename TS, typename TC, int V>
cudaError_t launch_update_sf(const TriSolve& M, const double* p, const double* q, double* x, double* r, double* z,
                             double* pp, double* part, PcgState* s, int mode, cudaStream_t st) {
  const size_t need = sf_smem_bytes(M.max_block, sizeof(TC));
  auto kern = k_pcg_update_sf<TS, TC, V>;
  SDSL_CUDA_TRY((allow_max_dynamic_smem<k_pcg_update_sf<TS, TC, V>>()));
  kern<<<(unsigned)M.nblocks, M.threads, need, st>>>(M, p, q, x, r, z, pp, part, s, mode); count_launch();
  return cudaGetLastError();
}

cudaError_t update_any(const TriSolve& M, const double* p, const double* q, double* x, double* r, double* z,
                       double* pp, double* part, PcgState* s, int mode, cudaStream_t st) {
  return by_lanes(M.lanes, [&](auto V) -> cudaError_t {
    constexpr int kV = decltype(V)::value;
    if (M.staged) return update_staged(M, p, q, x, r, z, pp, part, s, mode, st);
    if (M.sync_free) {
      if (M.prec == 64) return launch_update_sf<double, double, kV>(M, p, q, x, r, z, pp, part, s, mode, st);
      if (M.apply_prec == 64) return launch_update_sf<float, double, kV>(M, p, q, x, r, z, pp, part, s, mode, st);
      return launch_update_sf<float, float, kV>(M, p, q, x, r, z, pp, part, s, mode, st);
    }
    if (M.prec == 32) return launch_update<float, kV>(M, p, q, x, r, z, pp, part, s, mode, st);
    return launch_update<double, kV>(M, p, q, x, r, z, pp, part, s, mode, st);
  });
}

LongRows long_of(const SpmvPlan& A) {
  LongRows L;
  L.thr = A.n_long > 0 ? A.long_thr : 0;
  L.n = A.n_long;
  L.rows = A.long_rows;
  L.ax = A.long_ax;
  return L;
}

// Long rows of the plan (if any), one CTA each, before the row kernel.
cudaError_t long_rows(const SpmvPlan& A, const double* x, const PcgState* s, cudaStream_t st) {
  if (A.n_long <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(A.n_long, 152 * 8);
  k_long_dot<<<grid, kThreads, 0, st>>>(A.n_long, A.long_rows, A.rp, A.ci, A.v, x, A.long_ax, s); count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t spmv(const SpmvPlan& A, const double* x, double* y, cudaStream_t st) {
  return by_lanes(A.lanes, [&](auto V) -> cudaError_t {
    SDSL_CUDA_TRY(long_rows(A, x, nullptr, st));
    k_spmv<decltype(V)::value><<<A.grid, kThreads, 0, st>>>(A.n, A.rp, A.ci, A.v, x, y, long_of(A)); count_launch();
    return cudaGetLastError();
  });
}

// Mean device time of `reps` launches of the SpMV with the plan's lane width
// (the autotuner's probe; x and y are scratch vectors of length n).
cudaError_t time_spmv(const SpmvPlan& A, const double* x, double* y, int reps, float* ms, cudaStream_t st) {
  cudaEvent_t a, b;
  SDSL_CUDA_TRY(cudaEventCreate(&a));
  SDSL_CUDA_TRY(cudaEventCreate(&b));
  SDSL_CUDA_TRY(spmv(A, x, y, st));  // warm
  SDSL_CUDA_TRY(cudaEventRecord(a, st));
  for (int i = 0; i < reps; ++i) SDSL_CUDA_TRY(spmv(A, x, y, st));
  SDSL_CUDA_TRY(cudaEventRecord(b, st));
  SDSL_CUDA_TRY(cudaEventSynchronize(b));
  SDSL_CUDA_TRY(cudaEventElapsedTime(ms, a, b));
  *ms /= (float)reps;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return cudaSuccess;
}

cudaError_t factored_product(const SpmvPlan& A, const double* p, double* q, double* part, PcgState* s, int pcg,
                             cudaStream_t st) {
  if (A.sell) return sell_factored_product(A, p, q, part, s, pcg, st);
  SDSL_CUDA_TRY(by_lanes(A.at_lanes, [&](auto V) -> cudaError_t {
    k_at_theta<decltype(V)::value><<<A.at_grid, kThreads, 0, st>>>(A.ncols, A.at_rp, A.at_ci, A.at_v, A.theta, p, A.u,
                                                                   pcg ? s : nullptr); count_launch();
    return cudaGetLastError();
  }));
  return by_lanes(A.a_lanes, [&](auto V) -> cudaError_t {
    k_a_u_dot<decltype(V)::value><<<A.grid, kThreads, 0, st>>>(A.n, A.a_rp, A.a_ci, A.a_v, A.u, A.rho, p, q, part, s,
                                                               pcg); count_launch();
    return cudaGetLastError();
  });
}

// Resident CTAs per SM of a product kernel at a lane width (kind 0: k_spmv,
// 1: k_pcg_spmv, 2: k_at_theta, 3: k_a_u_dot), for one-wave grids.
int product_occupancy(int kind, int lanes) {
  int n = 0;
  by_lanes(lanes, [&](auto V) -> cudaError_t {
    constexpr int kV = decltype(V)::value;
    switch (kind) {
      case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_spmv<kV>, kThreads, 0);
      case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pcg_spmv<kV>, kThreads, 0);
      case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_at_theta<kV>, kThreads, 0);
      default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_a_u_dot<kV>, kThreads, 0);
    }
  });
  return n > 0 ? n : 1;
}

// Mean device time of each half of the factored product over `reps` launches
// (the autotuner's probe; p and q are scratch vectors).
cudaError_t time_factored(const SpmvPlan& A, const double* p, double* q, int reps, float* ms_at, float* ms_a,
                          cudaStream_t st) {
  cudaEvent_t ev[3];
  for (auto& e : ev) SDSL_CUDA_TRY(cudaEventCreate(&e));
  SDSL_CUDA_TRY(factored_product(A, p, q, nullptr, nullptr, 0, st));  // warm
  float t_at = 0.f, t_a = 0.f;
  for (int i = 0; i < reps; ++i) {
    SDSL_CUDA_TRY(cudaEventRecord(ev[0], st));
    SDSL_CUDA_TRY(by_lanes(A.at_lanes, [&](auto V) -> cudaError_t {
      k_at_theta<decltype(V)::value><<<A.at_grid, kThreads, 0, st>>>(A.ncols, A.at_rp, A.at_ci, A.at_v, A.theta, p,
                                                                     A.u, nullptr); count_launch();
      return cudaGetLastError();
    }));
    SDSL_CUDA_TRY(cudaEventRecord(ev[1], st));
    SDSL_CUDA_TRY(by_lanes(A.a_lanes, [&](auto V) -> cudaError_t {
      k_a_u_dot<decltype(V)::value><<<A.grid, kThreads, 0, st>>>(A.n, A.a_rp, A.a_ci, A.a_v, A.u, A.rho, p, q,
                                                                 nullptr, nullptr, 0); count_launch();
      return cudaGetLastError();
    }));
    SDSL_CUDA_TRY(cudaEventRecord(ev[2], st));
    SDSL_CUDA_TRY(cudaEventSynchronize(ev[2]));
    float a = 0.f, b = 0.f;
    SDSL_CUDA_TRY(cudaEventElapsedTime(&a, ev[0], ev[1]));
    SDSL_CUDA_TRY(cudaEventElapsedTime(&b, ev[1], ev[2]));
    t_at += a;
    t_a += b;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  *ms_at = t_at / (float)reps;
  *ms_a = t_a / (float)reps;
  return cudaSuccess;
}

cudaError_t pcg_spmv(const SpmvPlan& A, const double* p, double* q, double* part, PcgState* s, cudaStream_t st) {
  if (A.factored) return factored_product(A, p, q, part, s, 1, st);
  return by_lanes(A.lanes, [&](auto V) -> cudaError_t {
    SDSL_CUDA_TRY(long_rows(A, p, s, st));
    k_pcg_spmv<decltype(V)::value><<<A.grid, kThreads, 0, st>>>(A.n, A.rp, A.ci, A.v, p, q, part, s, long_of(A)); count_launch();
    return cudaGetLastError();
  });
}

cudaError_t pcg_update_precond(const TriSolve& M, const double* p, const double* q, double* x, double* r, double* z,
                               double* part, PcgState* s, cudaStream_t st) {
  return update_any(M, p, q, x, r, z, nullptr, part, s, 0, st);
}


size_t sf_smem_bytes(int64_t max_block, size_t tc_size) {
  return 2 * (((size_t)max_block * tc_size + 15) & ~(size_t)15);
}

cudaError_t precond_apply(const TriSolve& M, const double* r, double* z, double* p_out, double* part, PcgState* s,
                          int mode, cudaStream_t st) {
  return update_any(M, nullptr, nullptr, nullptr, const_cast<double*>(r), z, p_out, part, s, mode, st);
}

cudaError_t pcg_direction(int64_t n, const double* z, double* p, PcgState* s, cudaStream_t st) {
  k_pcg_direction<<<grid_for(n, kThreads), kThreads, 0, st>>>(n, z, p, s); count_launch();
  return cudaGetLastError();
}

int direction_grid(int64_t n) { return (int)grid_for(n, kThreads); }

cudaError_t batch_direction(const BatchReq* reqs, const BatchItem* items, int nitems, int grid, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  k_batch_direction<<<(unsigned)std::min(grid, nitems), kThreads, 0, st>>>(reqs, items, nitems); count_launch();
  return cudaGetLastError();
}

cudaError_t true_residual(const SpmvPlan& A, const double* b, const double* x, double* r, double* part,
                          PcgState* s, int write_r, cudaStream_t st) {
  return by_lanes(A.lanes, [&](auto V) -> cudaError_t {
    SDSL_CUDA_TRY(long_rows(A, x, nullptr, st));
    k_residual<decltype(V)::value><<<A.grid, kThreads, 0, st>>>(A.n, A.rp, A.ci, A.v, b, x, r, part, s, write_r,
                                                                long_of(A)); count_launch();
    return cudaGetLastError();
  });
}

cudaError_t norm2_sq(int64_t n, const double* a, double* part, double* out, unsigned int* ticket, cudaStream_t st) {
  const unsigned g = grid_for(n, kThreads, 152 * 4);
  k_norm2<<<g, kThreads, 0, st>>>(n, a, part, out, ticket); count_launch();
  return cudaGetLastError();
}

cudaError_t pcg_init_state(PcgState* s, double tol2, long long maxit, cudaStream_t st) {
  k_init_state<<<1, 1, 0, st>>>(s, tol2, maxit); count_launch();
  return cudaGetLastError();
}

}  // namespace sdsl
