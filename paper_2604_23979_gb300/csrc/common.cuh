// common.cuh -- shared device helpers of the sm_103a library (not the oracle).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sdsl {

constexpr int kWarp = 32;

#define SDSL_CUDA_TRY(expr)                         \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return _e;               \
  } while (0)

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over aligned groups of G lanes (G a power of two <= 32); every lane of a
// group ends with the group's sum.  Fixed butterfly order => deterministic.
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
  if (G > 1) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Deterministic block-wide sum of a double: warp butterflies, then warp 0 adds
// the warp totals in warp order.  Every thread must call it; the result is
// valid in thread 0.  `sh` needs blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const unsigned w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    const unsigned nw = (blockDim.x + 31) >> 5;
    for (unsigned i = 0; i < nw; ++i) t += sh[i];
  }
  return t;
}

// Sum a[0..n) in index order by one thread (the partial-sum arrays are short).
__device__ __forceinline__ double serial_sum(const double* a, int n) {
  double t = 0.0;
  for (int i = 0; i < n; ++i) t += a[i];
  return t;
}

// First index in sorted a[lo, hi) equal to key, or -1.
__device__ __forceinline__ int64_t bsearch_i32(const int32_t* __restrict__ a, int64_t lo, int64_t hi,
                                               int32_t key) {
  hi -= 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) >> 1;
    int32_t v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

// Allow a kernel the device's whole opt-in dynamic shared memory.  The limit
// is a property of the function, shared by every handle in the process: it is
// raised once per device and never lowered, so a launch captured in one
// handle's CUDA graph stays valid while other handles launch the same kernel
// with less.  (Occupancy follows the size each launch requests.)
inline cudaError_t set_max_dynamic_smem(const void* kern) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

template <auto Kern>
cudaError_t allow_max_dynamic_smem() {
  static int done[64] = {};  // per device; a racing second set is idempotent
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  e = set_max_dynamic_smem(reinterpret_cast<const void*>(Kern));
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = 1;
  return e;
}

// First index in sorted a[lo, hi) with a[index] >= key (hi if none).
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t* __restrict__ a, int64_t lo, int64_t hi,
                                                   int32_t key) {
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Process-wide count of kernel launches made by this library (every
// `<<<...>>>` launch site calls count_launch once per launch).
void count_launch(long long k = 1);
long long launches_so_far();

// Exclusive prefix sum (in place) of an int64 array of length n+1 whose first
// n entries are counts; entry n receives the total.  Three launches:
// chunk sums, scan of chunk sums, chunk-local scan.
cudaError_t exclusive_scan_i64(int64_t* data, int64_t n, int64_t* scratch, cudaStream_t st);
int64_t scan_scratch_elems(int64_t n);

// Exclusive scan of int32 counts into int32 offsets (out has n+1 entries).
cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st);

}  // namespace sdsl
