// dense_lu.cu -- blocked LU with partial pivoting of the dense border Schur
// complement (Sec. 2.4: S_B is dense and factored once per preconditioner
// build): FP32 storage, FP64 panels and pivots, the trailing update on the
// 5th-generation tensor cores.
//
// Right-looking, panels of kNb columns:
//   panel  (one CTA, FP64 on a widened copy of the panel): for each column,
//          pivot = largest |a_ik| (lowest i on ties), swap whole rows,
//          l_ik = a_ik / a_kk, rank-1 update of the panel's remaining
//          columns -- the unblocked algorithm on the panel; the pivots a_kk
//          are kept in FP64;
//   trsm   U12 = L11^{-1} A12 (unit lower L11, one thread per column);
//   update A22 -= L21 U12 as a tcgen05.mma GEMM (kind::tf32, accumulator in
//          tensor memory).  FP32 accuracy from TF32 inputs by splitting each
//          operand x = hi + lo (hi = tf32(x), lo = tf32(x - hi)) and summing
//          hi*hi + hi*lo + lo*hi in the FP32 accumulator.
// Output format as the unblocked kernels: LU in place (unit L below the
// diagonal, U on and above), ipiv[k] = row swapped with row k at step k.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace sdsl {

namespace {

constexpr int kNb = 64;        // panel width = K of the trailing GEMM
constexpr int kTile = 128;     // GEMM tile (M = N = 128) per CTA
constexpr int kPanelThreads = 1024;
constexpr int kSpinMax = 1 << 20;  // bounded mbarrier wait (try_wait itself may suspend briefly)

// ---------------------------------------------------------------- panel

// Columns [k0, k0 + kb), rows [k0, n); row swaps act on whole rows.
__global__ void __launch_bounds__(kPanelThreads) k_lu_panel(int64_t n, int64_t k0, int kb, float* __restrict__ A,
                                                            int32_t* __restrict__ ipiv, int* __restrict__ status) {
  __shared__ float bv[32];
  __shared__ int64_t bi[32];
  __shared__ int64_t piv;
  for (int j = 0; j < kb; ++j) {
    const int64_t k = k0 + j;
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
      for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
        const float t = A[k * n + c];
        A[k * n + c] = A[p * n + c];
        A[p * n + c] = t;
      }
    __syncthreads();
    const float pk = A[k * n + k];
    for (int64_t i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * n + k] = A[i * n + k] / pk;
    __syncthreads();
    // rank-1 update of the panel's columns right of k: thread (x, y) of a
    // 64 x 16 arrangement takes column k + 1 + x of rows k + 1 + y, y + 16, ...
    const int rem = kb - j - 1;
    const int tx = threadIdx.x & (kNb - 1), ty = threadIdx.x / kNb;
    if (tx < rem) {
      const int64_t c = k + 1 + tx;
      const float ukc = A[k * n + c];
      for (int64_t i = k + 1 + ty; i < n; i += kPanelThreads / kNb)
        A[i * n + c] = __fmaf_rn(-A[i * n + k], ukc, A[i * n + c]);
    }
    __syncthreads();
  }
}

// Panel in FP64 (the factorization's pivots): the panel's columns [k0, k0 +
// kb) of rows [k0, n) are widened into W (row i - k0, column j at
// W[(i - k0) * kNb + j]); pivot search (largest |w|, lowest row on ties),
// scaling by the pivot and the panel's rank-1 updates run in FP64, and the
// pivots are kept in FP64 (udiag[k]).  Row swaps act on W and, outside the
// panel's columns, on the FP32 matrix; at the end the panel's values are
// rounded back into it.  The trailing update (outside) stays FP32.
__global__ void __launch_bounds__(kPanelThreads) k_lu_panel64(int64_t n, int64_t k0, int kb, float* __restrict__ A,
                                                              double* __restrict__ W, double* __restrict__ udiag,
                                                              int32_t* __restrict__ ipiv, int* __restrict__ status) {
  __shared__ double bv[32];
  __shared__ int64_t bi[32];
  __shared__ int64_t piv;
  const int64_t rows = n - k0;
  for (int64_t t = threadIdx.x; t < rows * kb; t += blockDim.x) {
    const int64_t i = t / kb, j = t % kb;
    W[i * kNb + j] = (double)A[(k0 + i) * n + k0 + j];
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    const int64_t k = k0 + j;
    double best = -1.0;
    int64_t bidx = j;
    for (int64_t i = j + threadIdx.x; i < rows; i += blockDim.x) {
      const double v = fabs(W[i * kNb + j]);
      if (v > best) { best = v; bidx = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int64_t oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
    }
    if (lane_id() == 0) { bv[threadIdx.x >> 5] = best; bi[threadIdx.x >> 5] = bidx; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = -1.0;
      int64_t p = j;
      for (unsigned w = 0; w < blockDim.x / 32; ++w)
        if (bv[w] > b || (bv[w] == b && bi[w] < p)) { b = bv[w]; p = bi[w]; }
      piv = p;
      ipiv[k] = (int32_t)(k0 + p);
      if (!(b > 0.0) || !isfinite(b)) *status = 1;
    }
    __syncthreads();
    const int64_t p = piv;
    if (p != j) {
      for (int c = threadIdx.x; c < kb; c += blockDim.x) {
        const double t = W[j * kNb + c];
        W[j * kNb + c] = W[p * kNb + c];
        W[p * kNb + c] = t;
      }
      for (int64_t c = threadIdx.x; c < n - kb; c += blockDim.x) {  // columns outside the panel
        const int64_t cc = c < k0 ? c : c + kb;
        const float t = A[k * n + cc];
        A[k * n + cc] = A[(k0 + p) * n + cc];
        A[(k0 + p) * n + cc] = t;
      }
    }
    __syncthreads();
    const double pk = W[j * kNb + j];
    if (threadIdx.x == 0) udiag[k] = pk;
    for (int64_t i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) W[i * kNb + j] = W[i * kNb + j] / pk;
    __syncthreads();
    // rank-1 update, four rows per thread and round: all loads of a round
    // are issued before its stores (the loop over one array cannot be
    // reordered by the compiler otherwise)
    const int rem = kb - j - 1;
    const int tx = threadIdx.x & (kNb - 1), ty = threadIdx.x / kNb;
    constexpr int kRs = kPanelThreads / kNb;  // row stride: 16
    if (tx < rem) {
      const int c = j + 1 + tx;
      const double ukc = W[j * kNb + c];
      for (int64_t i0 = j + 1 + ty; i0 < rows; i0 += 4 * kRs) {
        double a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + u * kRs;
          a[u] = i < rows ? W[i * kNb + j] : 0.0;
          b[u] = i < rows ? W[i * kNb + c] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t i = i0 + u * kRs;
          if (i < rows) W[i * kNb + c] = __fma_rn(-a[u], ukc, b[u]);
        }
      }
    }
    __syncthreads();
  }
  for (int64_t t = threadIdx.x; t < rows * kb; t += blockDim.x) {
    const int64_t i = t / kb, j = t % kb;
    A[(k0 + i) * n + k0 + j] = (float)W[i * kNb + j];
  }
}

// ---------------------------------------------------------------- trsm

// A12 (rows [k0, k0+kb), columns [k0+kb, n)) := L11^{-1} A12, one column per
// thread, column-oriented: x_i -= l_ij x_j for j ascending (the same order of
// subtractions per entry as the row-oriented form).
constexpr int kTrsmThreads = 64;
__global__ void __launch_bounds__(kTrsmThreads) k_lu_trsm(int64_t n, int64_t k0, int kb, float* __restrict__ A) {
  __shared__ float L[kNb][kNb + 1];
  __shared__ float xs[kNb][kTrsmThreads];
  for (int t = threadIdx.x; t < kb * kb; t += blockDim.x) L[t / kb][t % kb] = A[(k0 + t / kb) * n + k0 + t % kb];
  const int64_t c = k0 + kb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = c < n;
  for (int i = 0; i < kb; ++i) xs[i][threadIdx.x] = valid ? A[(k0 + i) * n + c] : 0.f;
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    const float xj = xs[j][threadIdx.x];
    for (int i = j + 1; i < kb; ++i) xs[i][threadIdx.x] = __fmaf_rn(-L[i][j], xj, xs[i][threadIdx.x]);
  }
  if (valid)
    for (int i = 0; i < kb; ++i) A[(k0 + i) * n + c] = xs[i][threadIdx.x];
}

// ---------------------------------------------------------------- tcgen05 GEMM

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
// K-adjacent core matrices 128 B apart (leading byte offset), 8-row groups
// kLdSbo bytes apart (stride byte offset).  Element (r, k) of a 128 x kNb tile:
constexpr uint32_t kLbo = 128;
constexpr uint32_t kSbo = (kNb / 4) * 128;  // 2048
constexpr int kTileBytes = kTile / 8 * kSbo;  // 32 KiB
__device__ __forceinline__ int canon_off(int r, int k) {
  return (r >> 3) * kSbo + (k >> 2) * kLbo + (r & 7) * 16 + (k & 3) * 4;
}

// Shared-memory matrix descriptor (sm_100 family): start, leading and stride
// byte offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(kLbo >> 4) << 16;
  d |= (uint64_t)(kSbo >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major,
// N = 128, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTile >> 3) << 17) |
                            ((uint32_t)(kTile >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// C -= A B for row-major panels: A is M x kb (lda), B is kb x N (ldb), C is
// M x N (ldc), kb <= kNb.  The panels may lie in one array (disjoint regions).
struct GemmSub {
  const float* A;
  int64_t lda;
  const float* B;
  int64_t ldb;
  float* C;
  int64_t ldc;
  int64_t M, N;
  int kb;
};

// One 128 x 128 tile of C per CTA (4 warps): operands split into tf32 hi/lo
// in shared memory, 3 x 8 tcgen05.mma (K = 8 each) into a tensor-memory
// accumulator, then C -= accumulator.
__global__ void __launch_bounds__(128) k_gemm_sub_tc(GemmSub g, int* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int timed_out;
  unsigned char* Ah = smem;
  unsigned char* Al = smem + kTileBytes;
  unsigned char* Bh = smem + 2 * kTileBytes;
  unsigned char* Bl = smem + 3 * kTileBytes;
  const int64_t r0 = (int64_t)blockIdx.y * kTile;  // tile rows (M)
  const int64_t c0 = (int64_t)blockIdx.x * kTile;  // tile columns (N)
  const int warp = threadIdx.x >> 5, lane = lane_id();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_addr(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    timed_out = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // A: consecutive threads take consecutive k of a row; B: consecutive
  // columns of a row of B (both coalesced).  Zero outside the panels.
  for (int t = threadIdx.x; t < kTile * kNb; t += blockDim.x) {
    const int r = t / kNb, k = t % kNb;
    const int64_t gr = r0 + r;
    const float a = (gr < g.M && k < g.kb) ? g.A[gr * g.lda + k] : 0.f;
    const float ah = to_tf32(a);
    const int off = canon_off(r, k);
    *reinterpret_cast<float*>(Ah + off) = ah;
    *reinterpret_cast<float*>(Al + off) = to_tf32(a - ah);
  }
  for (int t = threadIdx.x; t < kTile * kNb; t += blockDim.x) {
    const int c = t % kTile, k = t / kTile;
    const int64_t gc = c0 + c;
    const float b = (gc < g.N && k < g.kb) ? g.B[(int64_t)k * g.ldb + gc] : 0.f;
    const float bh = to_tf32(b);
    const int off = canon_off(c, k);
    *reinterpret_cast<float*>(Bh + off) = bh;
    *reinterpret_cast<float*>(Bl + off) = to_tf32(b - bh);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (threadIdx.x == 0) {
    const uint32_t ah = smem_addr(Ah), al = smem_addr(Al), bh = smem_addr(Bh), bl = smem_addr(Bl);
    uint32_t acc = 0;
    // small cross terms first, then the leading term
    for (int s = 0; s < kNb / 8; ++s) {  // K = 8 tf32 per MMA = two core matrices
      const uint32_t o = (uint32_t)s * 2 * kLbo;
      mma_tf32(tmem, smem_desc(al + o), smem_desc(bh + o), acc);
      acc = 1;
      mma_tf32(tmem, smem_desc(ah + o), smem_desc(bl + o), 1);
    }
    for (int s = 0; s < kNb / 8; ++s) {
      const uint32_t o = (uint32_t)s * 2 * kLbo;
      mma_tf32(tmem, smem_desc(ah + o), smem_desc(bh + o), 1);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(&mbar))
                 : "memory");
  }
  // bounded wait for the MMAs (phase 0)
  bool done = false;
  for (int spin = 0; spin < kSpinMax && !done; ++spin) done = mbar_try(smem_addr(&mbar), 0);
  if (!done) {
    atomicExch(&timed_out, 1);
    *status = 2;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (!timed_out) {
    // epilogue: thread (warp, lane) owns tile row 32 warp + lane (TMEM lane)
    const int64_t gr = r0 + 32 * warp + lane;
    for (int cb = 0; cb < kTile; cb += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (gr < g.M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int64_t gc = c0 + cb + j;
          if (gc < g.N) g.C[gr * g.ldc + gc] -= __uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
  }
}

// The same update on CUDA cores (FP32 FMA, 32 x 32 tiles).
__global__ void k_gemm_sub_cc(GemmSub g) {
  __shared__ float As[32][kNb + 1];
  __shared__ float Bs[kNb][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int t = threadIdx.y * 32 + threadIdx.x; t < 32 * kNb; t += 32 * 32) {
    const int rr = t / kNb, k = t % kNb;
    As[rr][k] = (r0 + rr < g.M && k < g.kb) ? g.A[(r0 + rr) * g.lda + k] : 0.f;
    const int kk = t / 32, cc = t % 32;
    Bs[kk][cc] = (c0 + cc < g.N && kk < g.kb) ? g.B[(int64_t)kk * g.ldb + c0 + cc] : 0.f;
  }
  __syncthreads();
  const int64_t r = r0 + threadIdx.y, c = c0 + threadIdx.x;
  if (r >= g.M || c >= g.N) return;
  float s = 0.f;
  for (int k = 0; k < g.kb; ++k) s = __fmaf_rn(As[threadIdx.y][k], Bs[k][threadIdx.x], s);
  g.C[r * g.ldc + c] -= s;
}

cudaError_t gemm_sub(const GemmSub& g, int tensor_cores, int* status, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.kb <= 0) return cudaSuccess;
  if (tensor_cores) {
    const dim3 grid((unsigned)((g.N + kTile - 1) / kTile), (unsigned)((g.M + kTile - 1) / kTile));
    k_gemm_sub_tc<<<grid, 128, (size_t)4 * kTileBytes, st>>>(g, status); count_launch();
  } else {
    const dim3 grid((unsigned)((g.N + 31) / 32), (unsigned)((g.M + 31) / 32));
    k_gemm_sub_cc<<<grid, dim3(32, 32), 0, st>>>(g); count_launch();
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- inverse

// Y = P I: row i of Y is e_{perm(i)}, perm = the row swaps ipiv applied in order.
__global__ void k_perm_identity(int64_t n, const int32_t* __restrict__ ipiv, int32_t* __restrict__ perm) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t k = 0; k < n; ++k) {
      const int64_t p = ipiv[k];
      const int32_t t = perm[k];
      perm[k] = perm[p];
      perm[p] = t;
    }
  }
}

__global__ void k_fill_perm(int64_t n, const int32_t* __restrict__ perm, float* __restrict__ Y) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / n, j = t % n;
    Y[t] = (j == perm[i]) ? 1.f : 0.f;
  }
}

// Rows [i0, i0+kb) of X (n columns, row-major): X_I := T^{-1} X_I with T the
// diagonal block of LU at (i0, i0): unit lower (upper = 0) or upper with its
// diagonal (upper = 1).  One column per thread.
__global__ void __launch_bounds__(kTrsmThreads) k_trsm_block(int64_t n, const float* __restrict__ LU, int64_t i0,
                                                            int kb, float* __restrict__ X, int upper,
                                                            const double* __restrict__ udiag) {
  __shared__ float T[kNb][kNb + 1];
  __shared__ float xs[kNb][kTrsmThreads];
  for (int t = threadIdx.x; t < kb * kb; t += blockDim.x) T[t / kb][t % kb] = LU[(i0 + t / kb) * n + i0 + t % kb];
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = c < n;
  for (int i = 0; i < kb; ++i) xs[i][threadIdx.x] = valid ? X[(i0 + i) * n + c] : 0.f;
  __syncthreads();
  if (!upper) {
    for (int j = 0; j < kb; ++j) {
      const float xj = xs[j][threadIdx.x];
      for (int i = j + 1; i < kb; ++i) xs[i][threadIdx.x] = __fmaf_rn(-T[i][j], xj, xs[i][threadIdx.x]);
    }
  } else {
    for (int j = kb - 1; j >= 0; --j) {
      // the pivot in FP64 when the factorization kept it
      const float xj = udiag ? (float)((double)xs[j][threadIdx.x] / udiag[i0 + j]) : xs[j][threadIdx.x] / T[j][j];
      xs[j][threadIdx.x] = xj;
      for (int i = 0; i < j; ++i) xs[i][threadIdx.x] = __fmaf_rn(-T[i][j], xj, xs[i][threadIdx.x]);
    }
  }
  if (valid)
    for (int i = 0; i < kb; ++i) X[(i0 + i) * n + c] = xs[i][threadIdx.x];
}

}  // namespace

cudaError_t dense_lu_blocked(int64_t n, float* LU, int32_t* ipiv, double* W, double* udiag, int* status,
                             int tensor_cores, cudaStream_t st) {
  if (tensor_cores) SDSL_CUDA_TRY((allow_max_dynamic_smem<k_gemm_sub_tc>()));
  for (int64_t k0 = 0; k0 < n; k0 += kNb) {
    const int kb = (int)std::min<int64_t>(kNb, n - k0);
    if (W && udiag) {
      k_lu_panel64<<<1, kPanelThreads, 0, st>>>(n, k0, kb, LU, W, udiag, ipiv, status); count_launch();
    } else {
      k_lu_panel<<<1, kPanelThreads, 0, st>>>(n, k0, kb, LU, ipiv, status); count_launch();
    }
    SDSL_CUDA_TRY(cudaGetLastError());
    const int64_t rest = n - k0 - kb;
    if (rest <= 0) continue;
    k_lu_trsm<<<(unsigned)((rest + kTrsmThreads - 1) / kTrsmThreads), kTrsmThreads, 0, st>>>(n, k0, kb, LU); count_launch();
    SDSL_CUDA_TRY(cudaGetLastError());
    GemmSub g;  // A22 -= L21 U12
    g.A = LU + (k0 + kb) * n + k0;
    g.lda = n;
    g.B = LU + k0 * n + k0 + kb;
    g.ldb = n;
    g.C = LU + (k0 + kb) * n + k0 + kb;
    g.ldc = n;
    g.M = rest;
    g.N = rest;
    g.kb = kb;
    SDSL_CUDA_TRY(gemm_sub(g, tensor_cores, status, st));
  }
  return cudaSuccess;
}

// X = U^{-1} L^{-1} P from the blocked LU: forward block sweep with unit L,
// then backward with U; the block updates of the remaining rows are GEMMs.
cudaError_t dense_inverse_blocked(int64_t n, const float* LU, const int32_t* ipiv, const double* udiag, float* X,
                                  int32_t* perm, int* status, int tensor_cores, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (tensor_cores) SDSL_CUDA_TRY((allow_max_dynamic_smem<k_gemm_sub_tc>()));
  k_perm_identity<<<1, 32, 0, st>>>(n, ipiv, perm); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  k_fill_perm<<<(unsigned)std::min<int64_t>((n * n + 255) / 256, 152 * 16), 256, 0, st>>>(n, perm, X); count_launch();
  SDSL_CUDA_TRY(cudaGetLastError());
  const unsigned tgrid = (unsigned)((n + kTrsmThreads - 1) / kTrsmThreads);
  for (int64_t i0 = 0; i0 < n; i0 += kNb) {  // Y = L^{-1} P
    const int kb = (int)std::min<int64_t>(kNb, n - i0);
    k_trsm_block<<<tgrid, kTrsmThreads, 0, st>>>(n, LU, i0, kb, X, 0, nullptr); count_launch();
    SDSL_CUDA_TRY(cudaGetLastError());
    GemmSub g;  // rows below -= L[below, I] Y_I
    g.A = LU + (i0 + kb) * n + i0;
    g.lda = n;
    g.B = X + i0 * n;
    g.ldb = n;
    g.C = X + (i0 + kb) * n;
    g.ldc = n;
    g.M = n - i0 - kb;
    g.N = n;
    g.kb = kb;
    SDSL_CUDA_TRY(gemm_sub(g, tensor_cores, status, st));
  }
  const int64_t nblk = (n + kNb - 1) / kNb;
  for (int64_t b = nblk - 1; b >= 0; --b) {  // X = U^{-1} Y
    const int64_t i0 = b * kNb;
    const int kb = (int)std::min<int64_t>(kNb, n - i0);
    k_trsm_block<<<tgrid, kTrsmThreads, 0, st>>>(n, LU, i0, kb, X, 1, udiag); count_launch();
    SDSL_CUDA_TRY(cudaGetLastError());
    GemmSub g;  // rows above -= U[above, I] X_I
    g.A = LU + i0;
    g.lda = n;
    g.B = X + i0 * n;
    g.ldb = n;
    g.C = X;
    g.ldc = n;
    g.M = i0;
    g.N = n;
    g.kb = kb;
    SDSL_CUDA_TRY(gemm_sub(g, tensor_cores, status, st));
  }
  return cudaSuccess;
}

}  // namespace sdsl
