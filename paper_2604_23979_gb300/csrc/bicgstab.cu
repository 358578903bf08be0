// bicgstab.cu -- the vector steps of right-preconditioned BiCGSTAB, the
// Krylov method paired with Block Jacobi in Sec. 4.3 (van der Vorst 1992;
// right preconditioning as in Sec. 2.2).  One pass:
//   p  = r  (first pass) or r + beta (p - omega v)          k_bicg_direction
//   ph = M^{-1} p                                            staged apply, mode 2
//   v  = S ph                                                product
//   alpha = rho / (rt . v)                                   k_bicg_alpha
//   x += alpha ph, s = r - alpha v, sh = M^{-1} s, ||s||     staged update, mode 0
//   t  = S sh                                                product
//   omega = (t . s) / (t . t)                                k_bicg_omega
//   x += omega sh, r = s - omega t, rho' = rt . r, beta      k_bicg_finish
// Every reduction is a fixed-order two-stage sum (per-CTA partials, the last
// CTA to arrive adds them in CTA order), so a solve is bit-reproducible.  The
// scalars live on the device; the kernels return at once when the shared
// PcgState says the solve is done, so whole passes can be captured in a graph.
#include "pcg_common.cuh"

namespace sdsl {

namespace {

constexpr int kBicgThreads = 256;

inline unsigned bicg_grid(int64_t n) {
  int64_t g = (n + kBicgThreads - 1) / kBicgThreads;
  if (g > kBicgMaxCtas) g = kBicgMaxCtas;
  return (unsigned)(g < 1 ? 1 : g);
}

// rt = r, rho = r . r, and the per-restart scalars.
__global__ void __launch_bounds__(kBicgThreads) k_bicg_restart(int64_t n, const double* __restrict__ r,
                                                               double* __restrict__ rt, BicgScalars* __restrict__ c) {
  __shared__ double sh[kBicgThreads / 32];
  double loc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = r[i];
    rt[i] = ri;
    loc = __fma_rn(ri, ri, loc);
  }
  const double tot = block_sum(loc, sh);
  if (threadIdx.x == 0) c->part[blockIdx.x] = tot;
  if (last_block(&c->ticket)) {
    if (threadIdx.x < 32) {
      const double rr = warp_fixed_sum(c->part, gridDim.x);
      if (threadIdx.x == 0) {
        c->rho = rr;
        c->beta = 0.0;
        c->omega = 0.0;
        c->first = 1;
        c->ticket = 0;
      }
    }
  }
}

// p = r on the first pass after a (re)start, else p = r + beta (p - omega v)
// (each operation rounded on its own, no contraction).
__global__ void __launch_bounds__(kBicgThreads) k_bicg_direction(int64_t n, const double* __restrict__ r,
                                                                 const double* __restrict__ v, double* __restrict__ p,
                                                                 const PcgState* __restrict__ s,
                                                                 const BicgScalars* __restrict__ c) {
  if (s->done) return;
  const bool first = c->first != 0;
  const double beta = c->beta, omega = c->omega;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (first) p[i] = r[i];
    else p[i] = __dadd_rn(r[i], __dmul_rn(beta, __dsub_rn(p[i], __dmul_rn(omega, v[i]))));
  }
}

// alpha = rho / (rt . v); the pass is counted here.  Breakdown (done = 3) on
// rt . v = 0 or a non-finite value.
__global__ void __launch_bounds__(kBicgThreads) k_bicg_alpha(int64_t n, const double* __restrict__ rt,
                                                             const double* __restrict__ v, PcgState* __restrict__ s,
                                                             BicgScalars* __restrict__ c) {
  if (s->done) return;
  __shared__ double sh[kBicgThreads / 32];
  double loc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    loc = __fma_rn(rt[i], v[i], loc);
  const double tot = block_sum(loc, sh);
  if (threadIdx.x == 0) c->part[blockIdx.x] = tot;
  if (last_block(&c->ticket)) {
    if (threadIdx.x < 32) {
      const double rv = warp_fixed_sum(c->part, gridDim.x);
      if (threadIdx.x == 0) {
        c->rv = rv;
        s->iters += 1;
        if (rv == 0.0 || !isfinite(rv)) s->done = 3;
        else s->alpha = c->rho / rv;
        c->ticket = 0;
      }
    }
  }
}

// omega = (t . s) / (t . t); breakdown on t . t <= 0 or a non-finite value.
__global__ void __launch_bounds__(kBicgThreads) k_bicg_omega(int64_t n, const double* __restrict__ t,
                                                             const double* __restrict__ sv, PcgState* __restrict__ s,
                                                             BicgScalars* __restrict__ c) {
  if (s->done) return;
  __shared__ double sh[kBicgThreads / 32];
  double ts = 0.0, tt = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ti = t[i];
    ts = __fma_rn(ti, sv[i], ts);
    tt = __fma_rn(ti, ti, tt);
  }
  const double tsb = block_sum(ts, sh);
  const double ttb = block_sum(tt, sh);
  if (threadIdx.x == 0) {
    c->part[blockIdx.x] = tsb;
    c->part[kBicgMaxCtas + blockIdx.x] = ttb;
  }
  if (last_block(&c->ticket)) {
    if (threadIdx.x < 32) {
      const double tst = warp_fixed_sum(c->part, gridDim.x);
      const double ttt = warp_fixed_sum(c->part + kBicgMaxCtas, gridDim.x);
      if (threadIdx.x == 0) {
        c->ts = tst;
        c->tt = ttt;
        if (!(ttt > 0.0) || !isfinite(ttt) || !isfinite(tst)) s->done = 3;
        else c->omega = tst / ttt;
        c->ticket = 0;
      }
    }
  }
}

// x += omega sh, r = s - omega t (r holds s on entry), ||r||^2 and rt . r;
// last CTA: convergence of the recurrence (done = 1), the pass limit
// (done = 2), breakdown (done = 3), else beta and rho for the next pass.
__global__ void __launch_bounds__(kBicgThreads) k_bicg_finish(int64_t n, const double* __restrict__ sh_vec,
                                                              const double* __restrict__ t,
                                                              const double* __restrict__ rt, double* __restrict__ x,
                                                              double* __restrict__ r, PcgState* __restrict__ s,
                                                              BicgScalars* __restrict__ c) {
  if (s->done) return;
  __shared__ double sh[kBicgThreads / 32];
  const double omega = c->omega;
  double rr = 0.0, rtr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = __dadd_rn(x[i], __dmul_rn(omega, sh_vec[i]));
    const double ri = __dsub_rn(r[i], __dmul_rn(omega, t[i]));
    r[i] = ri;
    rr = __fma_rn(ri, ri, rr);
    rtr = __fma_rn(rt[i], ri, rtr);
  }
  const double rrb = block_sum(rr, sh);
  const double rtrb = block_sum(rtr, sh);
  if (threadIdx.x == 0) {
    c->part[blockIdx.x] = rrb;
    c->part[kBicgMaxCtas + blockIdx.x] = rtrb;
  }
  if (last_block(&c->ticket)) {
    if (threadIdx.x < 32) {
      const double rrt = warp_fixed_sum(c->part, gridDim.x);
      const double rtrt = warp_fixed_sum(c->part + kBicgMaxCtas, gridDim.x);
      if (threadIdx.x == 0) {
        s->rr = rrt;
        if (rrt <= s->tol2) {
          s->done = 1;
        } else if (s->iters >= c->maxit) {
          s->done = 2;
        } else if (rtrt == 0.0 || omega == 0.0 || !isfinite(rtrt) || !isfinite(omega)) {
          s->done = 3;
        } else {
          c->beta = (rtrt / c->rho) * (s->alpha / omega);
          c->rho = rtrt;
          c->first = 0;
        }
        c->ticket = 0;
      }
    }
  }
}

__global__ void k_bicg_init(BicgScalars* c, long long maxit) {
  BicgScalars t = {};
  t.maxit = maxit;
  t.part = c->part;
  *c = t;
}

}  // namespace

cudaError_t bicg_init(BicgScalars* c, long long maxit, cudaStream_t st) {
  k_bicg_init<<<1, 1, 0, st>>>(c, maxit); count_launch();
  return cudaGetLastError();
}

cudaError_t bicg_restart(int64_t n, const double* r, double* rt, BicgScalars* c, cudaStream_t st) {
  k_bicg_restart<<<bicg_grid(n), kBicgThreads, 0, st>>>(n, r, rt, c); count_launch();
  return cudaGetLastError();
}

cudaError_t bicg_direction(int64_t n, const double* r, const double* v, double* p, const PcgState* s,
                           const BicgScalars* c, cudaStream_t st) {
  k_bicg_direction<<<bicg_grid(n), kBicgThreads, 0, st>>>(n, r, v, p, s, c); count_launch();
  return cudaGetLastError();
}

cudaError_t bicg_alpha(int64_t n, const double* rt, const double* v, PcgState* s, BicgScalars* c, cudaStream_t st) {
  k_bicg_alpha<<<bicg_grid(n), kBicgThreads, 0, st>>>(n, rt, v, s, c); count_launch();
  return cudaGetLastError();
}

cudaError_t bicg_omega(int64_t n, const double* t, const double* sv, PcgState* s, BicgScalars* c, cudaStream_t st) {
  k_bicg_omega<<<bicg_grid(n), kBicgThreads, 0, st>>>(n, t, sv, s, c); count_launch();
  return cudaGetLastError();
}

cudaError_t bicg_finish(int64_t n, const double* sh, const double* t, const double* rt, double* x, double* r,
                        PcgState* s, BicgScalars* c, cudaStream_t st) {
  k_bicg_finish<<<bicg_grid(n), kBicgThreads, 0, st>>>(n, sh, t, rt, x, r, s, c); count_launch();
  return cudaGetLastError();
}

}  // namespace sdsl
