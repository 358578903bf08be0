// scan.cu -- exclusive prefix sums used to turn per-row counts into CSR row
// pointers (filtered pattern, normal-equation pattern, transposes).
#include "common.cuh"

namespace sdsl {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int64_t kChunk = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T* sh, T* total) {
  // inclusive warp scan
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    const unsigned nw = blockDim.x >> 5;
    T s = lane < nw ? sh[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= (unsigned)o) s += y;
    }
    if (lane < nw) sh[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  T warp_prefix = w == 0 ? T(0) : sh[w - 1];
  if (total) *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_prefix + x - v;
}

__global__ void k_chunk_sums(const int64_t* __restrict__ d, int64_t n, int64_t* __restrict__ sums) {
  __shared__ int64_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * kChunk;
  int64_t t = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
    if (i < n) t += d[i];
  }
  int64_t tot;
  block_exclusive_scan<int64_t>(t, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t* __restrict__ sums, int64_t nchunks, int64_t* __restrict__ d, int64_t n) {
  __shared__ int64_t sh[32];
  int64_t carry = 0;
  for (int64_t base = 0; base < nchunks; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < nchunks ? sums[i] : 0;
    int64_t tot;
    int64_t ex = block_exclusive_scan<int64_t>(v, sh, &tot);
    if (i < nchunks) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) d[n] = carry;
}

__global__ void k_chunk_scan(int64_t* __restrict__ d, int64_t n, const int64_t* __restrict__ sums) {
  __shared__ int64_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t t = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? d[base + k] : 0;
    t += v[k];
  }
  int64_t ex = block_exclusive_scan<int64_t>(t, sh, nullptr) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) d[base + k] = ex;
    ex += v[k];
  }
}

__global__ void k_scan_i32(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n) {
  __shared__ int32_t sh[32];
  int32_t carry = 0;
  for (int64_t base = 0; base < n; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int32_t v = i < n ? in[i] : 0;
    int32_t tot;
    int32_t ex = block_exclusive_scan<int32_t>(v, sh, &tot);
    if (i < n) out[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) out[n] = carry;
}

}  // namespace

int64_t scan_scratch_elems(int64_t n) { return (n + kChunk - 1) / kChunk + 1; }

cudaError_t exclusive_scan_i64(int64_t* data, int64_t n, int64_t* scratch, cudaStream_t st) {
  const int64_t nchunks = (n + kChunk - 1) / kChunk;
  if (nchunks > 0) {
    k_chunk_sums<<<(unsigned)nchunks, kScanThreads, 0, st>>>(data, n, scratch); count_launch();
    SDSL_CUDA_TRY(cudaGetLastError());
  }
  k_scan_sums<<<1, 1024, 0, st>>>(scratch, nchunks, data, n); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  if (nchunks > 0) {
    k_chunk_scan<<<(unsigned)nchunks, kScanThreads, 0, st>>>(data, n, scratch); count_launch();
    SDSL_CUDA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t st) {
  k_scan_i32<<<1, 1024, 0, st>>>(in, out, n); count_launch();
  return cudaGetLastError();
}

}  // namespace sdsl
