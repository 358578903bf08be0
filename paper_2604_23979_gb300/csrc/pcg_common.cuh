// pcg_common.cuh -- device helpers shared by the PCG kernels of krylov.cu
// (SpMV, level-synchronous and flag-free block solves) and sweep.cu (staged
// block solves): deterministic reductions, the update epilogue and the
// "not yet solved" sentinel of the flag-synchronised sweeps.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace sdsl {
namespace {

// Deterministic sum of a[0, n) by one warp (lane-strided, then butterfly).
__device__ __forceinline__ double warp_fixed_sum(const double* a, int n) {
  double t = 0.0;
  for (int i = lane_id(); i < n; i += 32) t += a[i];
  return warp_sum(t);
}

// Returns true in every thread of the last of `count` CTAs (or virtual CTAs
// of a batched launch) to arrive.
__device__ __forceinline__ bool last_block(unsigned int* ticket, unsigned count) {
  __shared__ int amlast;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) amlast = atomicAdd(ticket, 1u) == count - 1;
  __syncthreads();
  if (amlast) __threadfence();
  return amlast;
}
__device__ __forceinline__ bool last_block(unsigned int* ticket) { return last_block(ticket, gridDim.x); }

// Shared epilogue of the update kernels: z, the block partials of
// ||r||^2, r^T z and z^T q, and (last CTA) the scalars of the next launch.
// part holds three sections of nblocks entries: [rr | rz | zq].
// b: the block this CTA (or virtual CTA) solved; the request's M.nblocks
// CTAs take part in the reduction.
__device__ __forceinline__ void update_epilogue(const TriSolve& M, double rrb, double rzb, double zqb,
                                                double* __restrict__ part, PcgState* __restrict__ s, int mode,
                                                bool timed_out, int b) {
  const int nb = (int)M.nblocks;
  if (threadIdx.x == 0) {
    part[b] = rrb;
    part[nb + b] = rzb;
    part[2 * nb + b] = zqb;
    if (timed_out) s->err = 1;
  }
  if (mode >= 2) return;
  if (last_block(&s->ticket[2], (unsigned)nb)) {
    if (threadIdx.x < 32) {
      const double rrt = warp_fixed_sum(part, nb);
      const double rzt = warp_fixed_sum(part + nb, nb);
      const double zqt = warp_fixed_sum(part + 2 * nb, nb);
      if (threadIdx.x == 0) {
        s->rr = rrt;
        s->rz_new = rzt;
        s->zq = zqt;
        if (mode == 0) {
          if (rrt <= s->tol2) s->done = 1;
          else if (s->iters >= s->maxit) s->done = 2;
          else if (!isfinite(rzt) || !isfinite(rrt)) s->done = 3;
          // standard beta = rho_new / rho; flexible (Polak-Ribiere) beta =
          // z_new^T (r_new - r_old) / rho = -alpha z_new^T q / rho
          s->beta = M.flexible ? -s->alpha * zqt / s->rho : rzt / s->rho;
          s->rho = rzt;
        } else {
          s->rho = rzt;
        }
        s->ticket[2] = 0;
      }
    }
  }
}

constexpr int kSpinLimit = 1 << 26;
#ifndef SDSL_BACKOFF_NS
#define SDSL_BACKOFF_NS 20
#endif
constexpr unsigned kBackoffNs = SDSL_BACKOFF_NS;  // ~1 s of polling: a wait that long is a bug, reported as TIMEOUT

// "Not yet computed" marker of the flag-free sweeps: a signalling-NaN bit
// pattern.  Arithmetic never produces a signalling NaN (results are finite
// or the canonical quiet NaN), so a solved value can never look unsolved,
// and an aligned 32/64-bit shared-memory store publishes value and readiness
// at once -- no separate flag and no memory fence on the critical path.
__device__ __forceinline__ float sentinel(float) { return __uint_as_float(0x7FA5A5A5u); }
__device__ __forceinline__ double sentinel(double) { return __longlong_as_double(0x7FF4A5A5A5A5A5A5ll); }
__device__ __forceinline__ bool is_sentinel(float v) { return __float_as_uint(v) == 0x7FA5A5A5u; }
__device__ __forceinline__ bool is_sentinel(double v) { return __double_as_longlong(v) == 0x7FF4A5A5A5A5A5A5ll; }

}  // namespace
}  // namespace sdsl
