// api.cu -- the C ABI of include/sdsl.h: handle life cycle and host
// orchestration of the kernels (setup -> factor -> solve, update_diag).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <chrono>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "sdsl.h"

#include <atomic>

namespace sdsl {
static std::atomic<long long> g_launches{0};
void count_launch(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
sdsl_status report_error(sdsl_status s, const std::string& msg);
}  // namespace sdsl

using namespace sdsl;

namespace {

thread_local std::string g_err;

}  // namespace

// Error reporting for entry points defined in other translation units.
sdsl_status sdsl::report_error(sdsl_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

namespace {

sdsl_status fail(sdsl_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

sdsl_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SDSL_ERR_OOM : SDSL_ERR_CUDA;
}

#define TRY_CUDA(expr)                                   \
  do {                                                   \
    cudaError_t _e = (expr);                             \
    if (_e != cudaSuccess) return cuda_fail(_e, #expr);  \
  } while (0)

#define TRY(expr)                          \
  do {                                     \
    sdsl_status _s = (expr);               \
    if (_s != SDSL_OK) return _s;          \
  } while (0)

// Device allocations grouped by lifetime: `sys` lives until sdsl_free, `pc`
// is replaced at every preconditioner build.
struct Arena {
  std::vector<void*> ptrs;
  cudaStream_t st = nullptr;
  int64_t own = 0;               // bytes this arena holds
  int64_t* live = nullptr;       // the owner's running total and its peak (optional)
  int64_t* peak = nullptr;
  void track(int64_t* l, int64_t* p) { live = l; peak = p; }
  template <typename T>
  sdsl_status get(T** out, size_t count) {
    *out = nullptr;
    if (count == 0) count = 1;
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, count * sizeof(T), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    ptrs.push_back(p);
    *out = static_cast<T*>(p);
    own += (int64_t)(count * sizeof(T));
    if (live) {
      *live += (int64_t)(count * sizeof(T));
      if (peak && *live > *peak) *peak = *live;
    }
    return SDSL_OK;
  }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    ptrs.clear();
    if (live) *live -= own;
    own = 0;
  }
};

void ensure_pool(int dev) {
  static bool done[64] = {};
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;  // keep freed blocks for the next handle (serving, repeated setups)
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[dev] = true;
}

int pow2_lanes(double avg, double per_lane) {
  int l = 2;
  while (l < 32 && l * per_lane < avg) l <<= 1;
  return l;
}

}  // namespace

struct sdsl_handle_s {
  sdsl_options opt{};
  cudaStream_t st = nullptr;       // private stream (capturable)
  cudaStream_t user = nullptr;     // caller's stream, joined at entry/exit
  cudaEvent_t ev_a = nullptr, ev_b = nullptr, ev_join = nullptr;
  int dev = 0, sms = 152;
  long long graph_kernels = 0;     // kernels in one launch of the iteration graph
  // rows of the system matrix longer than long_thr (summed by one CTA each)
  bool long_planned = false;
  // sliced ELL copies of A and A^T (normal form): built once per handle
  bool sell_planned = false, sell_ok = false;
  SellMat a_sell{}, at_sell{};
  int long_thr = 0;
  int64_t n_long = 0;
  int32_t* long_rows = nullptr;
  double* long_ax = nullptr;
  int form = 0, method = 0;
  int64_t m = 0, n = 0, N = 0;  // input rows/cols, system dimension
  Arena sys, pc;
  int64_t live_bytes = 0, peak_bytes = 0;  // device memory held by the handle's arenas (and its peak)
  // input A (normal / augmented) and its transpose
  int64_t a_nnz = 0;
  int64_t *a_rp = nullptr, *at_rp = nullptr;
  int32_t *a_ci = nullptr, *at_ci = nullptr;
  double *a_v = nullptr, *at_v = nullptr, *theta = nullptr;
  // system matrix
  int64_t s_nnz = 0;
  int64_t* s_rp = nullptr;
  int32_t* s_ci = nullptr;
  double* s_v = nullptr;
  int64_t* xdiag = nullptr;  // augmented: position of every x diagonal
  // blocks
  int64_t nblocks = 0, border = 0;
  std::vector<int64_t> h_bp;  // interior blocks over the system rows
  int64_t* d_bp = nullptr;
  int32_t* row_block = nullptr;
  double* dvals = nullptr;
  // preconditioner
  int64_t p_nnz = 0;
  int64_t *p_rp = nullptr, *p_diag = nullptr, *mir = nullptr;
  int32_t* p_ci = nullptr;
  double *p_v = nullptr, *F = nullptr, *dinv = nullptr;
  float *Ff = nullptr, *dinvf = nullptr;
  std::vector<double> h_alpha;
  int32_t *lev_off_lo = nullptr, *lev_ptr_lo = nullptr, *lev_rows_lo = nullptr;
  int32_t *lev_off_up = nullptr, *lev_ptr_up = nullptr, *lev_rows_up = nullptr;
  std::vector<int32_t> h_nlev_lo, h_nlev_up;
  int32_t *row_lev_lo = nullptr, *row_lev_up = nullptr;  // level of every row within its block
  int64_t tot_lo = 0, tot_up = 0;
  // Krylov workspace
  double *b = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *u = nullptr;
  double *part = nullptr, *part_blk = nullptr, *scalars = nullptr;
  // BiCGSTAB: shadow residual, preconditioned direction, t = S M^{-1} s
  double *rt = nullptr, *ph = nullptr, *tv = nullptr;
  BicgScalars* bicg = nullptr;
  int64_t* scan_scratch = nullptr;
  int* flag = nullptr;
  PcgState* state = nullptr;
  PcgState* h_state = nullptr;  // pinned
  SpmvPlan A{};
  TriSolve M{};
  cudaGraphExec_t graph = nullptr;
  int graph_iters = 0;
  cudaEvent_t prof_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // BBD: border, dense Schur complement (FP64), its FP32 LU and inverse,
  // GMRES bases and apply scratch
  int64_t b0 = 0, nbord = 0;
  double* SB = nullptr;
  float *LU32 = nullptr, *Sinv = nullptr;
  int32_t* ipiv = nullptr;
  double* udiag = nullptr;  // FP64 pivots of the blocked LU (modes 0, 1)
  double *V = nullptr, *Z = nullptr, *bt = nullptr, *bg = nullptr, *bz = nullptr, *bres = nullptr, *bcor = nullptr;
  double *gpart = nullptr, *gh = nullptr;
  std::vector<int32_t> h_lev_off_lo, h_lev_off_up;
  // reuse bookkeeping (Sec. 3.4)
  bool factored = false, need_rebuild = false;
  int64_t iters_post_build = -1;   // iterations of the first converged solve after the last build
  int64_t solves_since_build = 0;
  // filter threshold schedule (Sec. 4.3): tau of the next build, IPM steps seen
  double tau_next = 0.0, tau_built = 0.0;
  int64_t ipm_step = 0;
  double* x0 = nullptr;            // the caller's initial guess, kept for a re-solve
  sdsl_stats stats{};
};

namespace {

// Block Jacobi (Sec. 2.3) under either Krylov method: the same IC(0)
// preconditioner, staged sweeps and product plans.
inline bool bj_method(const sdsl_handle h) { return h->method == SDSL_BJ_PCG || h->method == SDSL_BJ_BICGSTAB; }
inline bool bbd_method(int method) { return method == SDSL_BBD_GMRES || method == SDSL_BBD_GCR; }

struct Scope {  // join the caller's stream on entry and exit
  sdsl_handle h;
  explicit Scope(sdsl_handle hh) : h(hh) {
    cudaEventRecord(h->ev_join, h->user);
    cudaStreamWaitEvent(h->st, h->ev_join, 0);
  }
  ~Scope() {
    cudaEventRecord(h->ev_join, h->st);
    cudaStreamWaitEvent(h->user, h->ev_join, 0);
  }
};

sdsl_status sync(sdsl_handle h, const char* where) {
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_fail(e, where);
  return SDSL_OK;
}

template <typename T>
sdsl_status to_host(sdsl_handle h, T* dst, const T* src, size_t count) {
  if (count == 0) return SDSL_OK;
  TRY_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDefault, h->st));
  return SDSL_OK;
}

template <typename T>
sdsl_status to_dev(sdsl_handle h, T* dst, const T* src, size_t count) {
  if (count == 0) return SDSL_OK;
  TRY_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyDefault, h->st));
  return SDSL_OK;
}

float elapsed(sdsl_handle h) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev_a, h->ev_b);
  return ms;
}

// Scan counts[0..n) into row pointers in place (counts has n+1 entries) and
// return the total on the host.
sdsl_status scan_total(sdsl_handle h, int64_t* counts, int64_t n, int64_t* total) {
  TRY_CUDA(exclusive_scan_i64(counts, n, h->scan_scratch, h->st));
  TRY(to_host(h, total, counts + n, 1));
  return sync(h, "scan");
}

sdsl_status alloc_workspace(sdsl_handle h) {
  const int64_t N = h->N;
  TRY(h->sys.get(&h->b, N));
  TRY(h->sys.get(&h->x, N));
  TRY(h->sys.get(&h->x0, N));
  TRY(h->sys.get(&h->r, N));
  TRY(h->sys.get(&h->z, N));
  TRY(h->sys.get(&h->p, N));
  TRY(h->sys.get(&h->q, N));
  if (h->form == SDSL_FORM_NORMAL) TRY(h->sys.get(&h->u, h->n));
  TRY(h->sys.get(&h->part, 152 * 32 + 64));
  TRY(h->sys.get(&h->scalars, 16));
  TRY(h->sys.get(&h->state, 1));
  if (!h->h_state) TRY_CUDA(cudaMallocHost(&h->h_state, sizeof(PcgState)));
  if (h->method == SDSL_BJ_BICGSTAB) {
    TRY(h->sys.get(&h->rt, N));
    TRY(h->sys.get(&h->ph, N));
    TRY(h->sys.get(&h->tv, N));
    TRY(h->sys.get(&h->bicg, 1));
    BicgScalars c{};
    TRY(h->sys.get(&c.part, 2 * kBicgMaxCtas));
    TRY(to_dev(h, h->bicg, &c, 1));
    TRY(sync(h, "bicgstab scalars"));
  }
  TRY_CUDA(cudaMemsetAsync(h->part, 0, sizeof(double) * (152 * 32 + 64), h->st));
  TRY_CUDA(cudaMemsetAsync(h->state, 0, sizeof(PcgState), h->st));
  TRY_CUDA(cudaMemsetAsync(h->x, 0, sizeof(double) * (size_t)N, h->st));
  return SDSL_OK;
}

sdsl_status check_block_ptr(const int64_t* bp, int64_t nb, int64_t end) {
  if (!bp) return fail(SDSL_ERR_ARG, "block_ptr is NULL");
  if (bp[0] != 0) return fail(SDSL_ERR_ARG, "block_ptr[0] must be 0");
  for (int64_t k = 0; k < nb; ++k)
    if (bp[k + 1] < bp[k]) return fail(SDSL_ERR_ARG, "block_ptr must be non-decreasing");
  if (bp[nb] != end) return fail(SDSL_ERR_ARG, "block_ptr[nblocks] does not match the dimension");
  return SDSL_OK;
}

// Copy a CSR (rowptr/col/val in mem_space) to the device and validate it.
sdsl_status load_csr(sdsl_handle h, int64_t nrows, int64_t ncols, const int64_t* rowptr, const int32_t* col,
                     const double* val, int64_t** rp, int32_t** ci, double** v, int64_t* nnz) {
  if (!rowptr) return fail(SDSL_ERR_ARG, "rowptr is NULL");
  int64_t first = 0, last = 0;
  TRY_CUDA(cudaMemcpy(&first, rowptr, sizeof(int64_t), cudaMemcpyDefault));
  TRY_CUDA(cudaMemcpy(&last, rowptr + nrows, sizeof(int64_t), cudaMemcpyDefault));
  if (first != 0 || last < 0) return fail(SDSL_ERR_ARG, "rowptr[0] must be 0 and rowptr[n] >= 0");
  *nnz = last;
  if (last > 0 && (!col || !val)) return fail(SDSL_ERR_ARG, "col/val is NULL");
  if (last >= ((int64_t)1 << 40)) return fail(SDSL_ERR_ARG, "nnz too large");
  TRY(h->sys.get(rp, nrows + 1));
  TRY(h->sys.get(ci, last));
  TRY(h->sys.get(v, last));
  TRY(to_dev(h, *rp, rowptr, nrows + 1));
  TRY(to_dev(h, *ci, col, last));
  TRY(to_dev(h, *v, val, last));
  TRY_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), h->st));
  TRY_CUDA(check_csr(nrows, ncols, *rp, *ci, h->flag, h->st));
  int bad = 0;
  TRY(to_host(h, &bad, h->flag, 1));
  TRY(sync(h, "check_csr"));
  if (bad) return fail(SDSL_ERR_ARG, "CSR columns out of range or not strictly ascending in a row");
  return SDSL_OK;
}

sdsl_status transpose_input(sdsl_handle h) {
  TRY(h->sys.get(&h->at_rp, h->n + 1));
  TRY(h->sys.get(&h->at_ci, h->a_nnz));
  TRY(h->sys.get(&h->at_v, h->a_nnz));
  int64_t* cursor = nullptr;
  Arena tmp;
  tmp.st = h->st;
  tmp.track(&h->live_bytes, &h->peak_bytes);
  TRY(tmp.get(&cursor, h->n + 1));
  TRY_CUDA(transpose_csr(h->m, h->n, h->a_rp, h->a_ci, h->a_v, h->at_rp, h->at_ci, h->at_v, h->scan_scratch, h->st));
  TRY_CUDA(transpose_fill(h->m, h->n, h->a_rp, h->a_ci, h->a_v, h->at_rp, h->at_ci, h->at_v, cursor, h->st));
  tmp.release();
  return SDSL_OK;
}

sdsl_status form_normal(sdsl_handle h) {
  const int64_t m = h->m;
  TRY(h->sys.get(&h->s_rp, m + 1));
  int32_t* long_rows = nullptr;
  Arena tmp;
  tmp.st = h->st;
  tmp.track(&h->live_bytes, &h->peak_bytes);
  TRY(tmp.get(&long_rows, m));
  TRY_CUDA(normal_symbolic_count(m, h->a_rp, h->a_ci, h->at_rp, h->at_ci, h->s_rp, long_rows, h->flag + 1, h->st));
  int nlong = 0;
  TRY(to_host(h, &nlong, h->flag + 1, 1));
  TRY(sync(h, "symbolic count"));
  TRY_CUDA(cudaMemsetAsync(h->flag + 2, 0, sizeof(int), h->st));
  TRY_CUDA(normal_symbolic_long(false, nlong, long_rows, h->a_rp, h->a_ci, h->at_rp, h->at_ci, h->s_rp, nullptr,
                                h->flag + 2, h->st));
  TRY(scan_total(h, h->s_rp, m, &h->s_nnz));
  int err = 0;
  TRY(to_host(h, &err, h->flag + 2, 1));
  TRY(sync(h, "symbolic long"));
  if (err) { tmp.release(); return fail(SDSL_ERR_ARG, "a row of S has more than 16384 candidate entries"); }
  TRY(h->sys.get(&h->s_ci, h->s_nnz));
  TRY(h->sys.get(&h->s_v, h->s_nnz));
  TRY_CUDA(normal_symbolic_fill(m, h->a_rp, h->a_ci, h->at_rp, h->at_ci, h->s_rp, h->s_ci, h->st));
  TRY_CUDA(normal_symbolic_long(true, nlong, long_rows, h->a_rp, h->a_ci, h->at_rp, h->at_ci, h->s_rp, h->s_ci,
                                h->flag + 2, h->st));
  tmp.release();
  TRY_CUDA(normal_values(m, h->a_rp, h->a_ci, h->a_v, h->at_rp, h->at_ci, h->at_v, h->theta, h->opt.rho, h->s_rp,
                         h->s_ci, h->s_v, h->st));
  return SDSL_OK;
}

sdsl_status form_augmented(sdsl_handle h, const int64_t* rbp, const int64_t* cbp) {
  const int64_t m = h->m, n = h->n, nb = h->nblocks, N = m + n;
  std::vector<int64_t> kbp(nb + 1);
  kbp[0] = 0;
  for (int64_t k = 0; k < nb; ++k) kbp[k + 1] = kbp[k] + (cbp[k + 1] - cbp[k]) + (rbp[k + 1] - rbp[k]);
  h->h_bp = kbp;
  int64_t *d_rbp, *d_cbp, *pos;
  Arena tmp;
  tmp.st = h->st;
  tmp.track(&h->live_bytes, &h->peak_bytes);
  TRY(tmp.get(&d_rbp, nb + 1));
  TRY(tmp.get(&d_cbp, nb + 1));
  TRY(tmp.get(&pos, N));
  TRY(to_dev(h, d_rbp, rbp, nb + 1));
  TRY(to_dev(h, d_cbp, cbp, nb + 1));
  TRY(h->sys.get(&h->d_bp, nb + 1));
  TRY(to_dev(h, h->d_bp, kbp.data(), nb + 1));
  TRY_CUDA(bbd_positions(m, n, nb, d_rbp, d_cbp, h->d_bp, pos, h->st));
  TRY(h->sys.get(&h->s_rp, N + 1));
  TRY_CUDA(augmented_count(m, n, h->a_rp, h->at_rp, pos, h->s_rp, h->st));
  TRY(scan_total(h, h->s_rp, N, &h->s_nnz));
  TRY(h->sys.get(&h->s_ci, h->s_nnz));
  TRY(h->sys.get(&h->s_v, h->s_nnz));
  TRY(h->sys.get(&h->xdiag, n));
  TRY_CUDA(augmented_fill(m, n, h->a_rp, h->a_ci, h->a_v, h->at_rp, h->at_ci, h->at_v, h->theta, h->opt.rho, pos,
                          h->s_rp, h->s_ci, h->s_v, h->xdiag, h->st));
  tmp.release();
  return SDSL_OK;
}

int lanes_for(double avg) {  // about 12+ nonzeros per lane (FP64 instruction economy)
  int lanes = 2;
  while (lanes < 32 && lanes * 2 * 12.0 <= avg) lanes <<= 1;
  return lanes;
}

// Grids of the product kernels: at least 64 rows per CTA, at most one full
// wave (resident CTAs per SM x SMs, capped at 8 per SM -- the partial-sum
// arrays hold that many), so no CTA waits for a second wave.
int one_wave(int64_t rows, int sms, int per_sm) {
  const int64_t g = std::min<int64_t>((rows + 63) / 64, (int64_t)sms * std::min(per_sm, 8));
  return (int)std::max<int64_t>(1, g);
}

void set_product_grids(sdsl_handle h) {
  SpmvPlan& A = h->A;
  if (A.factored) {
    A.at_grid = one_wave(h->n, h->sms, product_occupancy(2, A.at_lanes));
    A.grid = one_wave(h->N, h->sms, product_occupancy(3, A.a_lanes));
  } else {
    A.grid = one_wave(h->N, h->sms, product_occupancy(1, A.lanes));
  }
}

void choose_spmv_plan(sdsl_handle h) {
  const double avg = h->N > 0 ? (double)h->s_nnz / (double)h->N : 1.0;
  // Normal equations: the PCG product S p can use the factored form
  // A (theta o (A^T p)) + rho p -- the same operator, 2 nnz(A) instead of
  // nnz(S) multiply-adds and HBM entries.  Auto picks it when it moves fewer
  // bytes; the explicit S stays for the filter and the true residual.
  const int form = h->opt.spmv_form;
  const bool can = h->form == SDSL_FORM_NORMAL && bj_method(h);
  const bool fewer = 2.0 * (double)h->a_nnz < (double)h->s_nnz;
  h->A.factored = can && (form == 2 || form == 3 || (form == 0 && fewer)) ? 1 : 0;
  h->A.sell = h->A.factored && h->sell_ok && (form == 3 || form == 0) ? 1 : 0;
  if (h->A.sell) {
    h->A.a_sell = h->a_sell;
    h->A.at_sell = h->at_sell;
    h->A.sell_at_grid = sell_grid_for(h->at_sell.nslices, h->sms * std::min(sell_occupancy(0), 8));
    h->A.sell_a_grid = sell_grid_for(h->a_sell.nslices, h->sms * std::min(sell_occupancy(1), 8));
  }
  if (h->A.factored) {
    h->A.ncols = h->n;
    h->A.a_rp = h->a_rp; h->A.a_ci = h->a_ci; h->A.a_v = h->a_v;
    h->A.at_rp = h->at_rp; h->A.at_ci = h->at_ci; h->A.at_v = h->at_v;
    h->A.theta = h->theta;
    h->A.rho = h->opt.rho;
    h->A.u = h->u;
    h->A.a_lanes = lanes_for(h->m > 0 ? (double)h->a_nnz / (double)h->m : 1.0);
    h->A.at_lanes = lanes_for(h->n > 0 ? (double)h->a_nnz / (double)h->n : 1.0);
  }
  h->A.n = h->N;
  h->A.rp = h->s_rp;
  h->A.ci = h->s_ci;
  h->A.v = h->s_v;
  h->A.lanes = lanes_for(avg);
  h->A.long_thr = h->long_thr;
  h->A.n_long = h->n_long;
  h->A.long_rows = h->long_rows;
  h->A.long_ax = h->long_ax;
  set_product_grids(h);
}

// ------------------------------------------------------------- autotuner
// Launch shapes picked by timing candidates on the handle's own matrix: the
// PCG product (explicit S at each lane width; the factored form on CSR, each
// half at each lane width; the factored form on the sliced ELL copies) and
// the staged sweeps' tile shape (entries per lane, far gap).  A choice is
// kept per structure (device, sizes of A and S, blocks, method, precisions)
// for the life of the process, so the first factorization of a structure
// pays the timing and later handles and rebuilds of it reuse the choice.  A
// candidate replaces the default only when it is at least 5 % faster, so
// close calls keep the same (default) arithmetic order.
struct TuneKey {
  int dev, method, fprec, aprec;
  int64_t N, a_nnz, s_nnz, nb;
  int64_t fixed;  // the options that narrow the candidates (packed): a choice is reused only under the same ones
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, method, fprec, aprec, N, a_nnz, s_nnz, nb, fixed) <
           std::tie(o.dev, o.method, o.fprec, o.aprec, o.N, o.a_nnz, o.s_nnz, o.nb, o.fixed);
  }
};
struct TuneChoice {
  int product = 0;  // 0 untuned, 1 explicit S, 2 factored CSR, 3 factored sliced ELL
  int lanes = 0, at_lanes = 0, a_lanes = 0;
  int E = 0, gap = 0;
  float ms = 0.f;  // time spent tuning
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice>& tune_cache() {
  static std::map<TuneKey, TuneChoice> m;
  return m;
}
TuneKey tune_key(sdsl_handle h, int apply) {
  const sdsl_options& o = h->opt;
  const int64_t fixed = (int64_t)o.sweep_lane_entries | (int64_t)o.sweep_far_gap << 8 | (int64_t)o.sweep_wait << 16 |
                        (int64_t)o.wait_test << 20 | (int64_t)o.spmv_form << 24 | (int64_t)o.sweep_slots << 28;
  return TuneKey{h->dev, h->method, h->opt.factor_prec, apply, h->N, h->a_nnz, h->s_nnz, h->nblocks, fixed};
}

// Mean device time of one call of `launch` (after one untimed call).
template <typename F>
sdsl_status time_calls(sdsl_handle h, int reps, float* ms, F launch) {
  TRY_CUDA(launch());
  cudaEvent_t a, b;
  TRY_CUDA(cudaEventCreate(&a));
  TRY_CUDA(cudaEventCreate(&b));
  cudaEventRecord(a, h->st);
  for (int i = 0; i < reps; ++i) {
    cudaError_t e = launch();
    if (e != cudaSuccess) { cudaEventDestroy(a); cudaEventDestroy(b); return cuda_fail(e, "tuning launch"); }
  }
  cudaEventRecord(b, h->st);
  cudaError_t e = cudaEventSynchronize(b);
  float t = 0.f;
  cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "tuning sync");
  *ms = t / (float)reps;
  return SDSL_OK;
}

cudaError_t product(sdsl_handle h, const double* y, double* out);

// Autotuner of the PCG product (see the autotuner notes above):
// explicit S at every lane width, the factored form on CSR (each half at
// every lane width), the factored form on the sliced ELL copies.
sdsl_status tune_product(sdsl_handle h) {
  const int form = h->opt.spmv_form;
  const bool can_factored = h->form == SDSL_FORM_NORMAL && bj_method(h);
  TRY_CUDA(cudaMemsetAsync(h->p, 0, sizeof(double) * (size_t)h->N, h->st));
  const SpmvPlan def = h->A;
  float def_ms = 1e30f;
  TRY(time_calls(h, 3, &def_ms, [&]() { return product(h, h->p, h->q); }));
  float best = def_ms;
  SpmvPlan best_plan = def;
  int best_kind = def.factored ? (def.sell ? 3 : 2) : 1;
  auto consider = [&](const SpmvPlan& P, int kind) -> sdsl_status {
    h->A = P;
    float ms = 1e30f;
    TRY(time_calls(h, 3, &ms, [&]() { return product(h, h->p, h->q); }));
    if (ms < best) { best = ms; best_plan = P; best_kind = kind; }
    return SDSL_OK;
  };
  if (form == 0 || form == 1) {  // explicit S
    SpmvPlan P = def;
    P.factored = 0;
    P.sell = 0;
    for (int l = 2; l <= 32; l <<= 1) {
      P.lanes = l;
      P.grid = one_wave(h->N, h->sms, product_occupancy(1, l));
      TRY(consider(P, 1));
    }
  }
  if (can_factored && (form == 0 || form == 2)) {  // factored on CSR: the halves' widths independently
    SpmvPlan P = def;
    P.factored = 1;
    P.sell = 0;
    P.ncols = h->n;
    P.a_rp = h->a_rp; P.a_ci = h->a_ci; P.a_v = h->a_v;
    P.at_rp = h->at_rp; P.at_ci = h->at_ci; P.at_v = h->at_v;
    P.theta = h->theta;
    P.rho = h->opt.rho;
    P.u = h->u;
    float b_at = 1e30f, b_a = 1e30f;
    int l_at = 4, l_a = 4;
    for (int l = 2; l <= 32; l <<= 1) {
      P.at_lanes = P.a_lanes = l;
      P.at_grid = one_wave(h->n, h->sms, product_occupancy(2, l));
      P.grid = one_wave(h->N, h->sms, product_occupancy(3, l));
      float ms_at = 0.f, ms_a = 0.f;
      TRY_CUDA(time_factored(P, h->p, h->q, 3, &ms_at, &ms_a, h->st));
      if (ms_at < b_at) { b_at = ms_at; l_at = l; }
      if (ms_a < b_a) { b_a = ms_a; l_a = l; }
    }
    P.at_lanes = l_at;
    P.a_lanes = l_a;
    P.at_grid = one_wave(h->n, h->sms, product_occupancy(2, l_at));
    P.grid = one_wave(h->N, h->sms, product_occupancy(3, l_a));
    TRY(consider(P, 2));
  }
  if (can_factored && h->sell_ok && (form == 0 || form == 3) && !def.sell) {
    SpmvPlan P = def;
    P.factored = 1;
    P.sell = 1;
    P.a_sell = h->a_sell;
    P.at_sell = h->at_sell;
    P.sell_at_grid = sell_grid_for(h->at_sell.nslices, h->sms * std::min(sell_occupancy(0), 8));
    P.sell_a_grid = sell_grid_for(h->a_sell.nslices, h->sms * std::min(sell_occupancy(1), 8));
    P.ncols = h->n;
    P.a_rp = h->a_rp; P.a_ci = h->a_ci; P.a_v = h->a_v;
    P.at_rp = h->at_rp; P.at_ci = h->at_ci; P.at_v = h->at_v;
    P.theta = h->theta;
    P.rho = h->opt.rho;
    P.u = h->u;
    TRY(consider(P, 3));
  }
  if (best > 0.95f * def_ms) { best_plan = def; best_kind = def.factored ? (def.sell ? 3 : 2) : 1; }
  h->A = best_plan;
  h->stats.tuned_spmv_lanes = best_kind == 1 ? best_plan.lanes : 0;
  h->stats.product_kind = best_kind;
  return SDSL_OK;
}

// The tuned product for this handle's structure: from the cache, or timed
// now and cached.
sdsl_status tune_spmv(sdsl_handle h) {
  const TuneKey key = tune_key(h, h->M.apply_prec);
  TuneChoice ch{};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) ch = it->second;
  }
  if (ch.product != 0) {
    SpmvPlan& A = h->A;
    if (ch.product == 1) {
      A.factored = 0;
      A.sell = 0;
      A.lanes = ch.lanes;
    } else {
      h->opt.spmv_form = ch.product;  // re-plan in that form with the tuned widths
      choose_spmv_plan(h);
      if (ch.product == 2) {
        A.at_lanes = ch.at_lanes;
        A.a_lanes = ch.a_lanes;
      }
    }
    set_product_grids(h);
    h->stats.product_kind = ch.product;
    return SDSL_OK;
  }
  auto t0 = std::chrono::steady_clock::now();
  TRY(tune_product(h));
  const float ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
  h->stats.ms_tune += ms;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  TuneChoice& c = tune_cache()[key];
  c.product = h->stats.product_kind;
  c.lanes = h->A.lanes;
  c.at_lanes = h->A.at_lanes;
  c.a_lanes = h->A.a_lanes;
  c.ms += ms;
  return SDSL_OK;
}

sdsl_status destroy_graph(sdsl_handle h) {
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return SDSL_OK;
}

// One PCG iteration = three launches (see krylov.cu).
sdsl_status enqueue_pcg_iteration(sdsl_handle h) {
  TRY_CUDA(pcg_spmv(h->A, h->p, h->q, h->part, h->state, h->st));
  TRY_CUDA(pcg_update_precond(h->M, h->p, h->q, h->x, h->r, h->z, h->part_blk, h->state, h->st));
  TRY_CUDA(pcg_direction(h->N, h->z, h->p, h->state, h->st));
  return SDSL_OK;
}

// The system product S y: factored (A (theta o (A^T y)) + rho y) or explicit.
cudaError_t product(sdsl_handle h, const double* y, double* out) {
  if (h->A.factored) return factored_product(h->A, y, out, nullptr, nullptr, 0, h->st);
  return spmv(h->A, y, out, h->st);
}

// The product of a BiCGSTAB pass: the factored form returns at once when the
// solve has stopped (the explicit form always runs).
cudaError_t pass_product(sdsl_handle h, const double* y, double* out) {
  if (h->A.factored) return factored_product(h->A, y, out, nullptr, h->state, 2, h->st);
  return spmv(h->A, y, out, h->st);
}

// One BiCGSTAB pass (bicgstab.cu).  The mode-0 PCG update computes
// x += alpha ph, s = r - alpha v (in r), sh = M^{-1} s (in z) and ||s||^2
// with its convergence test; v is kept in q.  Every kernel of a pass returns
// at once after the solve has stopped, so graphs of many passes waste little.
sdsl_status enqueue_bicg_iteration(sdsl_handle h) {
  const int64_t N = h->N;
  TRY_CUDA(bicg_direction(N, h->r, h->q, h->p, h->state, h->bicg, h->st));
  TRY_CUDA(precond_apply(h->M, h->p, h->ph, nullptr, h->part_blk, h->state, 3, h->st));
  TRY_CUDA(pass_product(h, h->ph, h->q));
  TRY_CUDA(bicg_alpha(N, h->rt, h->q, h->state, h->bicg, h->st));
  TRY_CUDA(pcg_update_precond(h->M, h->ph, h->q, h->x, h->r, h->z, h->part_blk, h->state, h->st));
  TRY_CUDA(pass_product(h, h->z, h->tv));
  TRY_CUDA(bicg_omega(N, h->tv, h->r, h->state, h->bicg, h->st));
  TRY_CUDA(bicg_finish(N, h->z, h->tv, h->rt, h->x, h->r, h->state, h->bicg, h->st));
  return SDSL_OK;
}

sdsl_status enqueue_iteration(sdsl_handle h) {
  return h->method == SDSL_BJ_BICGSTAB ? enqueue_bicg_iteration(h) : enqueue_pcg_iteration(h);
}

// Profile mode: one iteration with CUDA events around each kernel; the
// device times are accumulated into stats.kernel_ms / kernel_launches.
sdsl_status profiled_iteration(sdsl_handle h) {
  cudaEvent_t* e = h->prof_ev;
  TRY_CUDA(cudaEventRecord(e[0], h->st));
  TRY_CUDA(pcg_spmv(h->A, h->p, h->q, h->part, h->state, h->st));
  TRY_CUDA(cudaEventRecord(e[1], h->st));
  TRY_CUDA(pcg_update_precond(h->M, h->p, h->q, h->x, h->r, h->z, h->part_blk, h->state, h->st));
  TRY_CUDA(cudaEventRecord(e[2], h->st));
  TRY_CUDA(pcg_direction(h->N, h->z, h->p, h->state, h->st));
  TRY_CUDA(cudaEventRecord(e[3], h->st));
  TRY(sync(h, "profiled iteration"));
  for (int k = 0; k < 3; ++k) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e[k], e[k + 1]);
    h->stats.kernel_ms[k] += ms;
    h->stats.kernel_launches[k] += 1;
  }
  return SDSL_OK;
}

// Rows of the system matrix with more than max(1024, 16 x average) entries
// (the border rows of a BBD system span every block) get one CTA each in the
// products; the list depends only on the pattern, so it is built once.
sdsl_status plan_long_rows(sdsl_handle h) {
  if (h->long_planned) return SDSL_OK;
  const int64_t N = h->N;
  std::vector<int64_t> rp(N + 1);
  TRY(to_host(h, rp.data(), h->s_rp, N + 1));
  TRY(sync(h, "long rows"));
  const double avg = N > 0 ? (double)rp[N] / (double)N : 0.0;
  const int64_t thr = std::max<int64_t>(1024, (int64_t)(16.0 * avg));
  std::vector<int32_t> rows;
  for (int64_t i = 0; i < N; ++i)
    if (rp[i + 1] - rp[i] > thr) rows.push_back((int32_t)i);
  h->long_thr = (int)std::min<int64_t>(thr, INT32_MAX);
  h->n_long = (int64_t)rows.size();
  if (h->n_long > 0) {
    TRY(h->sys.get(&h->long_rows, h->n_long));
    TRY(h->sys.get(&h->long_ax, h->n_long));
    TRY(to_dev(h, h->long_rows, rows.data(), h->n_long));
  }
  h->long_planned = true;
  return SDSL_OK;
}

// SELL-32 copy of one CSR matrix; *ok = false (nothing kept) when padding
// would add more than 30 % to its entries.
sdsl_status build_sell(sdsl_handle h, int64_t nrows, const int64_t* rp, const int32_t* ci, const double* v,
                       int64_t nnz, SellMat* S, bool* ok) {
  *ok = false;
  const int64_t ns = (nrows + 31) / 32;
  int32_t *perm, *wid;
  int64_t* off;
  TRY(h->sys.get(&perm, std::max<int64_t>(ns * 32, 1)));
  TRY(h->sys.get(&wid, std::max<int64_t>(ns, 1)));
  TRY(h->sys.get(&off, ns + 1));
  Arena tmp;
  tmp.st = h->st;
  tmp.track(&h->live_bytes, &h->peak_bytes);
  struct Release {
    Arena& a;
    ~Release() { a.release(); }
  } release_tmp{tmp};
  int64_t* scratch;
  TRY(tmp.get(&scratch, scan_scratch_elems(ns) + 1));
  TRY_CUDA(sell_rank_widths(nrows, rp, perm, wid, off, h->st));
  TRY_CUDA(exclusive_scan_i64(off, ns, scratch, h->st));
  int64_t total = 0;
  TRY(to_host(h, &total, off + ns, 1));
  TRY(sync(h, "sell widths"));
  if ((double)total > 1.3 * (double)nnz + 32.0 * 64.0) return SDSL_OK;
  int32_t* col;
  double* val;
  TRY(h->sys.get(&col, std::max<int64_t>(total, 1)));
  TRY(h->sys.get(&val, std::max<int64_t>(total, 1)));
  TRY_CUDA(sell_fill(nrows, rp, ci, v, perm, off, wid, col, val, h->st));
  S->nrows = nrows;
  S->nslices = ns;
  S->perm = perm;
  S->off = off;
  S->wid = wid;
  S->col = col;
  S->val = val;
  *ok = true;
  return SDSL_OK;
}

sdsl_status plan_sell(sdsl_handle h) {
  if (h->sell_planned) return SDSL_OK;
  h->sell_planned = true;
  if (h->form != SDSL_FORM_NORMAL || !bj_method(h)) return SDSL_OK;
  if (h->opt.spmv_form == 1 || h->opt.spmv_form == 2) return SDSL_OK;
  bool ok_a = false, ok_at = false;
  TRY(build_sell(h, h->m, h->a_rp, h->a_ci, h->a_v, h->a_nnz, &h->a_sell, &ok_a));
  if (ok_a) TRY(build_sell(h, h->n, h->at_rp, h->at_ci, h->at_v, h->a_nnz, &h->at_sell, &ok_at));
  h->sell_ok = ok_a && ok_at;
  return SDSL_OK;
}

sdsl_status build_graph(sdsl_handle h) {
  destroy_graph(h);
  const int G = h->opt.graph_iters;
  if (G <= 0) return SDSL_OK;
  cudaGraph_t g = nullptr;
  const long long before = launches_so_far();
  TRY_CUDA(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed));
  sdsl_status s = SDSL_OK;
  for (int i = 0; i < G && s == SDSL_OK; ++i) s = enqueue_iteration(h);
  cudaError_t e = cudaStreamEndCapture(h->st, &g);
  h->graph_kernels = launches_so_far() - before;
  count_launch(-h->graph_kernels);  // captured, not executed: counted per graph launch
  if (s != SDSL_OK) { if (g) cudaGraphDestroy(g); return s; }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  h->graph_iters = G;
  return SDSL_OK;
}

sdsl_status build_levels(sdsl_handle h, int dir, int32_t** off, int32_t** ptr, int32_t** rows,
                         std::vector<int32_t>& nlev_h, int64_t* total, int32_t* cnt, int32_t* lev, int32_t* fa,
                         int32_t* fb, int32_t* nlev_d) {
  const int64_t nb = h->nblocks;
  TRY_CUDA(levels(dir, nb, h->d_bp, h->p_rp, h->p_ci, h->p_diag, cnt, lev, fa, fb, nlev_d, h->st));
  nlev_h.assign(nb, 0);
  TRY(to_host(h, nlev_h.data(), nlev_d, nb));
  TRY(sync(h, "levels"));
  std::vector<int32_t> off_h(nb + 1, 0);
  for (int64_t k = 0; k < nb; ++k) off_h[k + 1] = off_h[k] + nlev_h[k];
  *total = off_h[nb];
  TRY(h->pc.get(off, nb + 1));
  TRY(h->pc.get(ptr, *total + 1));
  TRY(h->pc.get(rows, h->h_bp[nb]));
  TRY(to_dev(h, *off, off_h.data(), nb + 1));
  const int32_t end = (int32_t)h->h_bp[nb];
  TRY(to_dev(h, *ptr + *total, &end, 1));
  TRY_CUDA(level_lists(nb, h->d_bp, lev, *off, cnt, *ptr, *rows, h->st));
  return sync(h, "level lists");
}

// BBD preconditioner (Sec. 2.4, third step): dense Schur complement of the
// border, its FP32 LU with partial pivoting and the explicit inverse.
sdsl_status build_bbd(sdsl_handle h) {
  const int64_t nb = h->nblocks, N = h->N;
  h->b0 = h->h_bp[nb];
  h->nbord = N - h->b0;
  const int64_t m = h->nbord;
  h->h_lev_off_lo.assign(nb + 1, 0);
  h->h_lev_off_up.assign(nb + 1, 0);
  for (int64_t k = 0; k < nb; ++k) {
    h->h_lev_off_lo[k + 1] = h->h_lev_off_lo[k] + h->h_nlev_lo[k];
    h->h_lev_off_up[k + 1] = h->h_lev_off_up[k] + h->h_nlev_up[k];
  }
  TRY(h->pc.get(&h->bt, N));
  TRY(h->pc.get(&h->bg, m + 1));
  TRY(h->pc.get(&h->bz, m + 1));
  TRY(h->pc.get(&h->bres, m + 1));
  TRY(h->pc.get(&h->bcor, m + 1));
  if (m == 0) return SDSL_OK;
  TRY(h->pc.get(&h->SB, m * m));
  TRY(h->pc.get(&h->LU32, m * m));
  TRY(h->pc.get(&h->Sinv, m * m));
  TRY(h->pc.get(&h->ipiv, m));
  TRY(h->pc.get(&h->udiag, m));
  TRY_CUDA(schur_init(m, h->b0, h->p_rp, h->p_ci, h->p_v, h->SB, h->st));
  Arena tmp;
  tmp.st = h->st;
  tmp.track(&h->live_bytes, &h->peak_bytes);
  float* work;
  // Waves of blocks assembled at once: every block writes its own dense
  // contribution, then the wave's contributions are subtracted from S_B in
  // block order -- the same per-entry order as one block at a time.  A wave
  // is bounded by the scratch it needs (about a quarter of free memory, at
  // most 6 GiB of solve scratch) and by 128 blocks.
  size_t free_b = 0, total_b = 0;
  TRY_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const int64_t tiles = schur_tiles(m);
  const size_t xcap = std::max<size_t>(std::min<size_t>(free_b / 4, (size_t)6 << 30), (size_t)1 << 20);
  const size_t ccap = std::max<size_t>(free_b / 8, (size_t)m * m * sizeof(double));
  std::vector<std::vector<SchurJob>> waves(1);
  size_t xw = 0;
  int64_t xmax = 0, jmax = 0;
  for (int64_t k = 0; k < nb; ++k) {
    const int64_t rows = h->h_bp[k + 1] - h->h_bp[k];
    const size_t xk = (size_t)tiles * rows * 32 * sizeof(double);
    auto& w = waves.back();
    if (!w.empty() && (xw + xk > xcap || w.size() >= 128 || (w.size() + 1) * (size_t)m * m * sizeof(double) > ccap)) {
      waves.emplace_back();
      xw = 0;
    }
    SchurJob J;
    J.s = h->h_bp[k];
    J.e = h->h_bp[k + 1];
    J.xoff = (int64_t)(xw / sizeof(double));
    J.L0 = h->h_lev_off_lo[k];
    J.L1 = h->h_lev_off_lo[k + 1];
    J.U0 = h->h_lev_off_up[k];
    J.U1 = h->h_lev_off_up[k + 1];
    waves.back().push_back(J);
    xw += xk;
    xmax = std::max<int64_t>(xmax, (int64_t)(xw / sizeof(double)));
    jmax = std::max<int64_t>(jmax, (int64_t)waves.back().size());
  }
  double *X, *Cpart;
  SchurJob* d_jobs;
  TRY(tmp.get(&X, (size_t)std::max<int64_t>(xmax, 1)));
  TRY(tmp.get(&Cpart, (size_t)jmax * m * m));
  TRY(tmp.get(&d_jobs, (size_t)nb));
  cudaEvent_t ev[4];
  for (auto& e : ev) TRY_CUDA(cudaEventCreate(&e));
  TRY_CUDA(cudaEventRecord(ev[0], h->st));
  int64_t jo = 0;
  for (const auto& w : waves) {  // waves in block order: deterministic accumulation
    if (w.empty()) continue;
    TRY(to_dev(h, d_jobs + jo, w.data(), w.size()));
    TRY_CUDA(schur_wave((int)w.size(), d_jobs + jo, h->b0, m, h->p_rp, h->p_ci, h->p_v, h->F, h->dinv, h->p_diag,
                        h->lev_ptr_lo, h->lev_rows_lo, h->lev_ptr_up, h->lev_rows_up, X, Cpart, h->SB, h->st));
    jo += (int64_t)w.size();
  }
  TRY_CUDA(cudaEventRecord(ev[1], h->st));
  TRY_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), h->st));
  double* W64;
  TRY(tmp.get(&W64, (size_t)m * 64));
  const bool blocked = h->opt.schur_lu != 2;
  TRY_CUDA(dense_lu_f32(m, h->SB, h->LU32, h->ipiv, blocked ? W64 : nullptr, blocked ? h->udiag : nullptr, h->flag,
                        h->opt.schur_lu, h->st));
  TRY_CUDA(cudaEventRecord(ev[2], h->st));
  TRY(tmp.get(&work, (size_t)m * ((m + 31) / 32) * 32));
  TRY_CUDA(dense_lu_inverse(m, h->LU32, h->ipiv, blocked ? h->udiag : nullptr, h->Sinv, work, h->opt.schur_lu,
                            h->flag, h->st));
  TRY_CUDA(cudaEventRecord(ev[3], h->st));
  int bad = 0;
  TRY(to_host(h, &bad, h->flag, 1));
  TRY(sync(h, "schur lu"));
  float t0 = 0.f, t1 = 0.f, t2 = 0.f;
  cudaEventElapsedTime(&t0, ev[0], ev[1]);
  cudaEventElapsedTime(&t1, ev[1], ev[2]);
  cudaEventElapsedTime(&t2, ev[2], ev[3]);
  h->stats.ms_schur = t0;
  h->stats.ms_dense_lu = t1;
  h->stats.ms_dense_inverse = t2;
  for (auto& e : ev) cudaEventDestroy(e);
  tmp.release();
  if (bad == 2) return fail(SDSL_ERR_TIMEOUT, "tensor-core update of the border Schur LU did not complete");
  if (bad) return fail(SDSL_ERR_BREAKDOWN, "zero pivot in the LU of the border Schur complement");
  return SDSL_OK;
}

// z = M^{-1} r for the BBD preconditioner (Sec. 2.4, fourth step).  The
// border solve uses the FP32 inverse of S_B with FP64 iterative refinement
// against the FP64 S_B (at most 10 steps, until ||g - S_B z_B|| <= 1e-12 ||g||).
sdsl_status bbd_apply(sdsl_handle h, const double* r, double* z) {
  const int64_t b0 = h->b0, m = h->nbord, nb = h->nblocks;
  TRY_CUDA(copy_vec(b0, r, h->bt, h->st));
  TRY_CUDA(block_lu_solve(nb, h->d_bp, h->p_rp, h->p_ci, h->F, h->dinv, h->p_diag, h->lev_off_lo, h->lev_ptr_lo,
                          h->lev_rows_lo, h->lev_off_up, h->lev_ptr_up, h->lev_rows_up, h->bt, h->st));
  if (m > 0) {
    TRY_CUDA(border_gather(m, b0, h->p_rp, h->p_ci, h->p_v, r, h->bt, h->bg, h->st));
    TRY_CUDA(dense_mv(m, h->Sinv, nullptr, h->bg, nullptr, h->bz, 0, h->st));
    double* nrm = h->scalars + 4;
    TRY_CUDA(norm2_sq(m, h->bg, h->part, nrm + 1, reinterpret_cast<unsigned int*>(h->part + 152 * 32), h->st));
    for (int it = 0; it < 10; ++it) {
      TRY_CUDA(dense_mv(m, nullptr, h->SB, h->bz, h->bg, h->bres, 1, h->st));
      TRY_CUDA(norm2_sq(m, h->bres, h->part, nrm, reinterpret_cast<unsigned int*>(h->part + 152 * 32), h->st));
      double hn[2];
      TRY(to_host(h, hn, nrm, 2));
      TRY(sync(h, "refinement"));
      if (!(hn[0] > 1e-24 * hn[1])) break;
      TRY_CUDA(dense_mv(m, h->Sinv, nullptr, h->bres, nullptr, h->bcor, 0, h->st));
      TRY_CUDA(axpy(m, 1.0, h->bcor, h->bz, h->st));
    }
  }
  TRY_CUDA(border_scatter(b0, h->p_rp, h->p_ci, h->p_diag, h->p_v, r, h->bz, z, h->st));
  TRY_CUDA(block_lu_solve(nb, h->d_bp, h->p_rp, h->p_ci, h->F, h->dinv, h->p_diag, h->lev_off_lo, h->lev_ptr_lo,
                          h->lev_rows_lo, h->lev_off_up, h->lev_ptr_up, h->lev_rows_up, z, h->st));
  if (m > 0) TRY_CUDA(copy_vec(m, h->bz, z + b0, h->st));
  return SDSL_OK;
}

// Right-preconditioned restarted GMRES(m) (Sec. 2.2): K M^{-1} u = b,
// x = M^{-1} u; classical Gram-Schmidt applied twice (CGS2) on the device,
// Hessenberg least squares with Givens rotations on the host.  The count is
// the number of Arnoldi steps (products K z).  Convergence on |g_{j+1}| <=
// rtol ||b||, confirmed by the true residual at the end of every cycle.
sdsl_status gmres_solve(sdsl_handle h) {
  const int64_t N = h->N;
  const int mres = std::max(1, h->opt.restart);
  sdsl_stats& S = h->stats;
  S.iters = 0;
  S.restarts = 0;
  double* bn2 = h->scalars;
  TRY_CUDA(norm2_sq(N, h->b, h->part, bn2, reinterpret_cast<unsigned int*>(h->part + 152 * 32), h->st));
  double bnorm2 = 0.0;
  TRY(to_host(h, &bnorm2, bn2, 1));
  TRY(sync(h, "gmres init"));
  if (bnorm2 == 0.0) {
    TRY_CUDA(cudaMemsetAsync(h->x, 0, sizeof(double) * (size_t)N, h->st));
    S.rel_res_true = S.rel_res_rec = 0.0;
    S.status = SDSL_OK;
    return SDSL_OK;
  }
  const double bnorm = std::sqrt(bnorm2), tol = h->opt.rtol * bnorm;
  std::vector<double> H((size_t)(mres + 1) * mres), cs(mres), sn(mres), g(mres + 1), y(mres), hv(mres + 2);
  SpmvPlan A = h->A;
  A.factored = 0;
  double* hdev = h->gh;
  int64_t it = 0;
  double gres = 0.0, tnorm = 0.0;
  sdsl_status result = SDSL_ERR_NOT_CONVERGED;
  for (;;) {
    TRY_CUDA(pcg_init_state(h->state, 0.0, 0, h->st));
    TRY_CUDA(true_residual(A, h->b, h->x, h->r, h->part, h->state, 1, h->st));
    TRY(to_host(h, h->h_state, h->state, 1));
    TRY(sync(h, "gmres residual"));
    tnorm = std::sqrt(h->h_state->tr);
    gres = tnorm;
    if (tnorm <= tol) { result = SDSL_OK; break; }
    if (it >= h->opt.maxit) break;
    S.restarts += 1;
    double* nrm = h->scalars + 1;
    {
      const double tb = tnorm;
      TRY(to_dev(h, nrm, &tb, 1));
    }
    TRY_CUDA(scale_to(N, nrm, 1, h->r, h->V, h->st));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = tnorm;
    int jend = 0;
    for (int j = 0; j < mres; ++j) {
      double* vj = h->V + (int64_t)j * N;
      double* zj = h->Z + (int64_t)j * N;
      double* w = h->V + (int64_t)(j + 1) * N;
      TRY(bbd_apply(h, vj, zj));
      TRY_CUDA(spmv(A, zj, w, h->st));
      ++it;
      if (h->opt.orthog == 1) {
        // CGS2: two passes of classical Gram-Schmidt against v_0 .. v_j
        TRY_CUDA(multidot(N, j + 1, h->V, N, w, h->gpart, hdev, h->st));
        TRY_CUDA(sub_multi(N, j + 1, h->V, N, hdev, w, h->st));
        TRY_CUDA(multidot(N, j + 1, h->V, N, w, h->gpart, hdev + mres + 1, h->st));
        TRY_CUDA(sub_multi(N, j + 1, h->V, N, hdev + mres + 1, w, h->st));
        TRY_CUDA(norm2_sq(N, w, h->part, hdev + 2 * (mres + 1), reinterpret_cast<unsigned int*>(h->part + 152 * 32),
                          h->st));
      } else {
        // modified Gram-Schmidt (the oracle's order): h_i = (w - sum_{l<i} h_l v_l)^T v_i
        for (int i = 0; i <= j; ++i)
          TRY_CUDA(mgs_step(N, w, i ? h->V + (int64_t)(i - 1) * N : nullptr, hdev + i - 1, h->V + (int64_t)i * N,
                            h->gpart, hdev + i, h->st));
        TRY_CUDA(mgs_step(N, w, h->V + (int64_t)j * N, hdev + j, nullptr, h->gpart, hdev + 2 * (mres + 1), h->st));
        TRY_CUDA(cudaMemsetAsync(hdev + mres + 1, 0, sizeof(double) * (size_t)(mres + 1), h->st));
      }
      std::vector<double> hh(2 * (mres + 1) + 1);
      TRY(to_host(h, hh.data(), hdev, 2 * (mres + 1) + 1));
      TRY(sync(h, "arnoldi"));
      const double hn = std::sqrt(hh[2 * (mres + 1)]);
      for (int i = 0; i <= j; ++i) H[(size_t)i * mres + j] = hh[i] + hh[mres + 1 + i];
      H[(size_t)(j + 1) * mres + j] = hn;
      if (hn != 0.0) {
        const double inv = hn;
        TRY(to_dev(h, nrm, &inv, 1));
        TRY_CUDA(scale_to(N, nrm, 1, w, w, h->st));
      }
      for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * mres + j], c = H[(size_t)(i + 1) * mres + j];
        H[(size_t)i * mres + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * mres + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[(size_t)j * mres + j], c = H[(size_t)(j + 1) * mres + j];
      const double rr = std::hypot(a, c);
      cs[j] = rr == 0.0 ? 1.0 : a / rr;
      sn[j] = rr == 0.0 ? 0.0 : c / rr;
      H[(size_t)j * mres + j] = rr;
      H[(size_t)(j + 1) * mres + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      gres = std::fabs(g[j + 1]);
      jend = j + 1;
      if (gres <= tol || it >= h->opt.maxit || hn == 0.0) break;
    }
    for (int i = jend - 1; i >= 0; --i) {
      double acc = g[i];
      for (int l = i + 1; l < jend; ++l) acc -= H[(size_t)i * mres + l] * y[l];
      y[i] = acc / H[(size_t)i * mres + i];
    }
    TRY(to_dev(h, hdev, y.data(), jend));
    TRY_CUDA(add_multi(N, jend, h->Z, N, hdev, h->x, h->st));
  }
  S.iters = it;
  S.restarts = std::max<int64_t>(0, S.restarts - 1);
  S.rel_res_true = tnorm / bnorm;
  S.rel_res_rec = gres / bnorm;
  S.status = result;
  if (result == SDSL_OK) return SDSL_OK;
  return fail(result, "GMRES reached maxit before the tolerance");
}

// Restarted right-preconditioned GCR(m) with the BBD preconditioner (the
// paper's IGCR(m), Sec. 4.2-4.3).  A cycle starts from the true residual;
// step j: p_j = M^{-1} r, q_j = K p_j; q_j is orthogonalised against the
// cycle's q_0 .. q_{j-1} by modified Gram-Schmidt (a chain of mgs_step, each
// coefficient taken after the previous subtraction), the same coefficients
// are subtracted from p_j, and both are divided by ||q_j||; then
// x += (q_j^T r) p_j, r -= (q_j^T r) q_j.  q_j lives in V, p_j in Z.
sdsl_status gcr_solve(sdsl_handle h) {
  const int64_t N = h->N;
  const int m = std::max(1, h->opt.restart);
  sdsl_stats& S = h->stats;
  S.iters = 0;
  S.restarts = 0;
  unsigned int* ticket = reinterpret_cast<unsigned int*>(h->part + 152 * 32);
  double* bn2 = h->scalars;
  TRY_CUDA(norm2_sq(N, h->b, h->part, bn2, ticket, h->st));
  double bnorm2 = 0.0;
  TRY(to_host(h, &bnorm2, bn2, 1));
  TRY(sync(h, "gcr init"));
  if (bnorm2 == 0.0) {
    TRY_CUDA(cudaMemsetAsync(h->x, 0, sizeof(double) * (size_t)N, h->st));
    S.rel_res_true = S.rel_res_rec = 0.0;
    S.status = SDSL_OK;
    return SDSL_OK;
  }
  const double bnorm = std::sqrt(bnorm2), tol = h->opt.rtol * bnorm;
  SpmvPlan A = h->A;
  A.factored = 0;
  double* c = h->gh;              // the step's Gram-Schmidt coefficients c_0 .. c_{j-1}
  double* d2 = h->gh + m;         // ||q_j||^2
  double* al = h->gh + m + 1;     // q_j^T r
  double* rn2 = h->gh + m + 2;    // ||r||^2
  double* dn = h->scalars + 1;    // ||q_j||, the divisor
  int64_t it = 0;
  double rnorm = 0.0, tnorm = 0.0;
  bool fresh = false;  // tnorm belongs to the current x
  sdsl_status result = SDSL_ERR_NOT_CONVERGED;
  for (;;) {
    TRY_CUDA(pcg_init_state(h->state, 0.0, 0, h->st));
    TRY_CUDA(true_residual(A, h->b, h->x, h->r, h->part, h->state, 1, h->st));
    TRY(to_host(h, h->h_state, h->state, 1));
    TRY(sync(h, "gcr residual"));
    tnorm = rnorm = std::sqrt(h->h_state->tr);
    fresh = true;
    if (tnorm <= tol) { result = SDSL_OK; break; }
    if (it >= h->opt.maxit) break;
    S.restarts += 1;
    bool breakdown = false;
    for (int j = 0; j < m && it < h->opt.maxit; ++j) {
      double* pj = h->Z + (int64_t)j * N;
      double* qj = h->V + (int64_t)j * N;
      TRY(bbd_apply(h, h->r, pj));
      TRY_CUDA(spmv(A, pj, qj, h->st));
      ++it;
      fresh = false;
      for (int i = 0; i < j; ++i)
        TRY_CUDA(mgs_step(N, qj, i ? h->V + (int64_t)(i - 1) * N : nullptr, i ? c + i - 1 : nullptr,
                          h->V + (int64_t)i * N, h->gpart, c + i, h->st));
      TRY_CUDA(mgs_step(N, qj, j ? h->V + (int64_t)(j - 1) * N : nullptr, j ? c + j - 1 : nullptr, nullptr,
                        h->gpart, d2, h->st));
      if (j > 0) TRY_CUDA(sub_multi(N, j, h->Z, N, c, pj, h->st));
      double dd = 0.0;
      TRY(to_host(h, &dd, d2, 1));
      TRY(sync(h, "gcr norm"));
      const double d = std::sqrt(dd);
      if (!(d > 0.0) || !std::isfinite(d)) { breakdown = true; break; }
      TRY(to_dev(h, dn, &d, 1));
      TRY_CUDA(scale_to(N, dn, 1, qj, qj, h->st));
      TRY_CUDA(scale_to(N, dn, 1, pj, pj, h->st));
      TRY_CUDA(multidot(N, 1, qj, N, h->r, h->gpart, al, h->st));
      TRY_CUDA(add_multi(N, 1, h->Z + (int64_t)j * N, N, al, h->x, h->st));
      TRY_CUDA(sub_multi(N, 1, qj, N, al, h->r, h->st));
      TRY_CUDA(norm2_sq(N, h->r, h->part, rn2, ticket, h->st));
      double r2 = 0.0;
      TRY(to_host(h, &r2, rn2, 1));
      TRY(sync(h, "gcr step"));
      rnorm = std::sqrt(r2);
      if (rnorm <= tol) break;
    }
    if (breakdown) { result = SDSL_ERR_BREAKDOWN; break; }
  }
  if (!fresh) {  // the true residual of the final iterate
    TRY_CUDA(pcg_init_state(h->state, 0.0, 0, h->st));
    TRY_CUDA(true_residual(A, h->b, h->x, h->r, h->part, h->state, 0, h->st));
    TRY(to_host(h, h->h_state, h->state, 1));
    TRY(sync(h, "gcr final residual"));
    tnorm = std::sqrt(h->h_state->tr);
  }
  S.iters = it;
  S.restarts = std::max<int64_t>(0, S.restarts - 1);
  S.rel_res_true = tnorm / bnorm;
  S.rel_res_rec = rnorm / bnorm;
  S.status = result;
  if (result == SDSL_OK) return SDSL_OK;
  if (result == SDSL_ERR_BREAKDOWN) return fail(result, "GCR breakdown: a direction with zero or non-finite norm");
  return fail(result, "GCR reached maxit before the tolerance");
}

// Variable-width tile streams of the staged sweeps (both directions).
// Rows of one level are packed into 32-lane tiles, each row with V lanes
// (the smallest power of two with E*V >= its entry count, at most 32, E the
// entries-per-lane target), in order of decreasing V so that groups sit at
// V-aligned lane offsets.  A tile is closed early when it would outgrow the
// ring slot.  The ring depth (4, 3 or 2 slots per warp) is the deepest whose
// slots hold the largest tile within the shared-memory budget.
// Returns SDSL_OK with *ok = false if the staging does not fit in shared
// memory (the caller then uses another solve kernel).
sdsl_status build_vtiles(sdsl_handle h, bool f32, int apply, int E, int gap, Arena& out, bool* ok) {
  TriSolve& M = h->M;
  const int64_t nb = h->nblocks;
  const int64_t nrows = h->h_bp[nb];
  const int tprec = h->opt.factor_prec == 16 ? 16 : f32 ? 32 : 64;  // stored value size: 2, 4 or 8 bytes
  const int tsz = tprec / 8;
  const int tc = apply == 32 ? 4 : 8;
  M.far_gap = gap;
  const int kWarps = 16;
  *ok = false;
  int64_t maxb = 0;
  for (int64_t k = 0; k < nb; ++k) maxb = std::max(maxb, h->h_bp[k + 1] - h->h_bp[k]);
  if (maxb > 65535) return SDSL_OK;  // block-local rows and columns are 16-bit
  struct Plan {
    std::vector<int32_t> trp{0}, rows;
    std::vector<int8_t> logv;
    std::vector<int64_t> toff{0}, tile_ptr;
    std::vector<int32_t> meta;  // per tile: level within the block, tiles of the two levels below
    int64_t max_bytes = 0;
  } plan[2];
  std::vector<int32_t> lptr[2], lrows[2];
  std::vector<int64_t> lens[2];
  int64_t* d_len;
  Arena tmp;
  tmp.st = h->st;
  tmp.track(&h->live_bytes, &h->peak_bytes);
  struct Release {
    Arena& a;
    ~Release() { a.release(); }
  } release_tmp{tmp};
  TRY(tmp.get(&d_len, nrows + 1));
  int* d_bad;
  TRY(tmp.get(&d_bad, 1));
  TRY_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), h->st));
  for (int dir = 0; dir < 2; ++dir) {
    const int64_t tot = dir == 0 ? h->tot_lo : h->tot_up;
    const int32_t* d_rows = dir == 0 ? h->lev_rows_lo : h->lev_rows_up;
    lptr[dir].resize(tot + 1);
    lrows[dir].resize(nrows);
    lens[dir].resize(nrows);
    TRY(to_host(h, lptr[dir].data(), dir == 0 ? h->lev_ptr_lo : h->lev_ptr_up, tot + 1));
    TRY(to_host(h, lrows[dir].data(), d_rows, nrows));
    TRY_CUDA(pack_count(dir, nrows, h->row_block, h->d_bp, h->p_rp, h->p_ci, h->p_diag, d_rows, d_len, h->st));
    TRY(to_host(h, lens[dir].data(), d_len, nrows));  // entry count of level position q
    TRY(sync(h, "tile plan"));
    for (int64_t q = 0; q < nrows; ++q)
      if (lens[dir][q] > 255 * 32) return SDSL_OK;  // a lane's entry count is 8-bit
  }
  auto tile_bytes = [&](int64_t nr, int64_t ne) {
    return 16 + 256 + ((nr * tsz + 15) & ~15) + ((2 * ne + 15) & ~15) + ((ne * tsz + 15) & ~15);
  };
  // Pack every level of every block into tiles no larger than cap bytes
  // (a single row larger than cap gets a tile of its own).
  auto make_plan = [&](int64_t cap) {
    for (int dir = 0; dir < 2; ++dir) {
      const std::vector<int32_t>& nl = dir == 0 ? h->h_nlev_lo : h->h_nlev_up;
      Plan& P = plan[dir];
      P = Plan{};
      P.tile_ptr.assign(nb + 1, 0);
      std::vector<std::pair<int, int32_t>> lev;  // (-logV, position)
      int64_t L = 0, tiles = 0;
      for (int64_t k = 0; k < nb; ++k) {
        P.tile_ptr[k] = tiles;
        std::vector<int32_t> lt;  // tiles of each level of this block so far
        for (int32_t l = 0; l < nl[k]; ++l, ++L) {
          const int64_t level_first = tiles;
          lev.clear();
          for (int32_t q = lptr[dir][L]; q < lptr[dir][L + 1]; ++q) {
            int lv = 0;
            while (lv < 5 && ((int64_t)E << lv) < lens[dir][q]) ++lv;
            lev.emplace_back(-lv, q);
          }
          std::stable_sort(lev.begin(), lev.end(), [](const std::pair<int, int32_t>& x,
                                                      const std::pair<int, int32_t>& y) { return x.first < y.first; });
          int used = 0, nr = 0;
          int64_t ne = 0;
          auto close = [&]() {
            if (nr == 0) return;
            const int64_t bytes = tile_bytes(nr, ne);
            P.toff.push_back(P.toff.back() + bytes);
            P.trp.push_back((int32_t)P.rows.size());
            P.max_bytes = std::max(P.max_bytes, bytes);
            P.meta.push_back(l);
            P.meta.push_back(l >= 1 ? lt[l - 1] : 0);
            P.meta.push_back(l >= gap ? lt[l - gap] : 0);
            ++tiles;
            nr = 0;
            ne = 0;
            used = 0;
          };
          for (const auto& e : lev) {
            const int V = 1 << (-e.first);
            const int64_t len = lens[dir][e.second];
            if (used + V > 32 || (nr > 0 && tile_bytes(nr + 1, ne + len) > cap)) close();
            P.rows.push_back(lrows[dir][e.second]);
            P.logv.push_back((int8_t)(-e.first));
            used += V;
            ++nr;
            ne += len;
          }
          close();
          lt.push_back((int32_t)(tiles - level_first));
        }
      }
      P.tile_ptr[nb] = tiles;
    }
  };
  auto max_tiles = [&]() {
    int64_t mt = 0;
    for (int64_t k = 0; k < nb; ++k)
      mt = std::max<int64_t>(mt, (plan[0].tile_ptr[k + 1] - plan[0].tile_ptr[k]) +
                                     (plan[1].tile_ptr[k + 1] - plan[1].tile_ptr[k]));
    return mt;
  };
  const size_t budget = (size_t)225 * 1024;
  int64_t maxlev = 0;
  for (int64_t k = 0; k < nb; ++k) maxlev = std::max<int64_t>(maxlev, std::max(h->h_nlev_lo[k], h->h_nlev_up[k]));
  make_plan(INT64_MAX);
  int64_t mt = max_tiles();
  const int64_t big = ((std::max(plan[0].max_bytes, plan[1].max_bytes) + 255) / 256) * 256;
  int slots = 0, slot = 0;
  const int forced = h->opt.sweep_slots;  // 0: the deepest ring that fits
  for (int sl = forced ? forced : 4; sl >= (forced ? forced : 2) && slots == 0; --sl)
    if (staged_smem_bytes(maxb, tc, kWarps, (int)big, sl, mt, maxlev) <= budget) { slots = sl; slot = (int)big; }
  if (slots == 0) {
    // the largest tiles do not fit the ring: cap the tiles at the largest
    // slot that does (the cap raises the tile count, so re-check)
    slots = forced ? forced : 2;
    const size_t fixed = staged_smem_bytes(maxb, tc, kWarps, 0, 0, 2 * mt, maxlev);
    if (fixed >= budget) return SDSL_OK;
    slot = (int)std::min<int64_t>(((budget - fixed) / ((size_t)kWarps * slots)) & ~(size_t)255, 16384);
    if (slot < 1024) return SDSL_OK;
    make_plan(slot);
    mt = max_tiles();
    if (staged_smem_bytes(maxb, tc, kWarps, slot, slots, mt, maxlev) > budget) return SDSL_OK;
  }
  M.slot_bytes = slot;
  M.slots = slots;
  M.max_tiles = mt;
  M.kreg = E <= 8 ? 8 : 16;
  M.max_levels = (int)maxlev;
  // per-value readiness where asked for; otherwise gap 1 (every entry far)
  // is the level-synchronous sweep and a larger gap the per-level barriers
  M.level_wait = h->opt.sweep_wait == 1 ? 0 : gap == 1 ? 2 : 1;
  // tiles of every level, in the order of the level offsets (block, level)
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<int32_t> lt, le;
    const Plan& P = plan[dir];
    const std::vector<int32_t>& nl = dir == 0 ? h->h_nlev_lo : h->h_nlev_up;
    int64_t t = 0;
    for (int64_t k = 0; k < nb; ++k) {
      for (int32_t l = 0; l < nl[k]; ++l) {
        int32_t c = 0;
        while (t < P.tile_ptr[k + 1] && P.meta[3 * t] == l) { ++c; ++t; }
        lt.push_back(std::max<int32_t>(c, 1));
        le.push_back((int32_t)(t - P.tile_ptr[k]));
      }
    }
    int32_t *d_lt, *d_le;
    TRY(out.get(&d_lt, lt.size()));
    TRY(out.get(&d_le, le.size()));
    TRY(to_dev(h, d_lt, lt.data(), lt.size()));
    TRY(to_dev(h, d_le, le.data(), le.size()));
    if (dir == 0) { M.fwd_ltiles = d_lt; M.fwd_lend = d_le; } else { M.bwd_ltiles = d_lt; M.bwd_lend = d_le; }
  }
  for (int dir = 0; dir < 2; ++dir) {
    Plan& P = plan[dir];
    const int64_t ntiles = (int64_t)P.trp.size() - 1;
    int32_t *d_trp, *d_rows;
    int8_t* d_logv;
    int64_t *d_toff, *d_tile;
    int32_t* d_meta;
    unsigned char* stream;
    TRY(out.get(&d_trp, ntiles + 1));
    TRY(out.get(&d_rows, P.rows.size()));
    TRY(out.get(&d_logv, P.logv.size()));
    TRY(out.get(&d_toff, ntiles + 1));
    TRY(out.get(&d_tile, nb + 1));
    TRY(tmp.get(&d_meta, P.meta.size()));
    TRY(out.get(&stream, P.toff.back()));
    TRY(to_dev(h, d_trp, P.trp.data(), ntiles + 1));
    TRY(to_dev(h, d_rows, P.rows.data(), P.rows.size()));
    TRY(to_dev(h, d_logv, P.logv.data(), P.logv.size()));
    TRY(to_dev(h, d_toff, P.toff.data(), ntiles + 1));
    TRY(to_dev(h, d_tile, P.tile_ptr.data(), nb + 1));
    TRY(to_dev(h, d_meta, P.meta.data(), P.meta.size()));
    TRY_CUDA(vt_fill(dir, ntiles, d_trp, d_rows, d_logv, h->row_block, h->d_bp, h->p_rp, h->p_ci, h->p_diag, h->F,
                     h->dinv, dir == 0 ? h->row_lev_lo : h->row_lev_up, tprec, d_toff, d_meta, stream,
                     d_bad, gap, h->st));
    if (dir == 0) { M.fwd_stream = stream; M.fwd_toff = d_toff; M.fwd_tile = d_tile; }
    else { M.bwd_stream = stream; M.bwd_toff = d_toff; M.bwd_tile = d_tile; }
  }
  int bad = 0;
  TRY(to_host(h, &bad, d_bad, 1));
  TRY(sync(h, "tile streams"));
  if (bad) return SDSL_OK;  // a row with more near entries than a lane record holds: another solve kernel
  *ok = true;
  return SDSL_OK;
}

// Tile shape of the staged sweeps: build each candidate's tile streams in a
// scratch arena and time the preconditioner apply (3 calls each).
sdsl_status tune_sweep(sdsl_handle h, bool f32, int apply, int* E_out, int* gap_out) {
  // Candidates (E, gap): gap >= 2 runs the per-level barrier protocol with
  // that far/near split, gap 1 the level-synchronous sweep (every entry far),
  // which is timed only when asked for (sweep_wait 3): on the staircase
  // workloads it loses to the barrier protocol at every shape.
  const int E0 = h->opt.sweep_lane_entries, G0 = h->opt.sweep_far_gap, W0 = h->opt.sweep_wait;
  std::vector<std::pair<int, int>> cand;
  if (W0 != 3) {
    const int Es[] = {16, 12, 24, 32};
    const int Gs[] = {3, 2, 4};
    for (int e : Es)
      for (int g : Gs)
        if ((E0 == 0 || e == E0) && (G0 == 0 || g == G0)) cand.emplace_back(e, g);
    if (cand.empty()) cand.emplace_back(E0 > 0 ? E0 : 16, G0 > 0 ? G0 : 3);
  }
  if (W0 == 3) {
    const int Es[] = {8, 4, 16, 2};
    for (int e : Es)
      if (E0 == 0 || e == E0) cand.emplace_back(e, 1);
    if (E0 != 0 && cand.empty()) cand.emplace_back(E0, 1);
  }
  TRY_CUDA(cudaMemsetAsync(h->r, 0, sizeof(double) * (size_t)h->N, h->st));
  float best = 1e30f, def = 1e30f;
  int bE = cand[0].first, bG = cand[0].second;
  for (size_t c = 0; c < cand.size(); ++c) {
    Arena tmp;
    tmp.st = h->st;
    tmp.track(&h->live_bytes, &h->peak_bytes);
    bool ok = false;
    sdsl_status s = build_vtiles(h, f32, apply, cand[c].first, cand[c].second, tmp, &ok);
    float ms = 1e30f;
    if (s == SDSL_OK && ok)
      s = time_calls(h, 3, &ms, [&]() {
        return precond_apply(h->M, h->r, h->z, nullptr, h->part_blk, h->state, 2, h->st);
      });
    tmp.release();
    TRY(s);
    if (c == 0) def = ms;
    if (ms < best) { best = ms; bE = cand[c].first; bG = cand[c].second; }
  }
  if (best > 0.95f * def) { bE = cand[0].first; bG = cand[0].second; }
  *E_out = bE;
  *gap_out = bG;
  return SDSL_OK;
}

sdsl_status factor_impl(sdsl_handle h) {
  h->stats.ms_tune = 0.0;
  cudaEventRecord(h->ev_a, h->st);
  h->pc.release();
  destroy_graph(h);
  h->factored = false;
  const int64_t N = h->N, nb = h->nblocks;
  const int whole = bbd_method(h->method) ? 1 : 0;
  // Eq. (filter) + Eq. (diagcorr)
  TRY_CUDA(diag_values(N, h->s_rp, h->s_ci, h->s_v, h->dvals, h->st));
  TRY(h->pc.get(&h->p_rp, N + 1));
  const double tau = h->tau_next;
  TRY_CUDA(filter_count(N, h->s_rp, h->s_ci, h->s_v, h->dvals, h->row_block, h->d_bp, whole, tau, h->p_rp,
                        h->st));
  TRY(scan_total(h, h->p_rp, N, &h->p_nnz));
  TRY(h->pc.get(&h->p_ci, h->p_nnz));
  TRY(h->pc.get(&h->p_v, h->p_nnz));
  TRY(h->pc.get(&h->p_diag, N));
  TRY(h->pc.get(&h->F, h->p_nnz));
  TRY(h->pc.get(&h->dinv, N));
  TRY(h->pc.get(&h->mir, h->p_nnz));
  TRY_CUDA(filter_fill(N, h->s_rp, h->s_ci, h->s_v, h->dvals, h->row_block, h->d_bp, whole, tau, h->opt.delta,
                       h->p_rp, h->p_ci, h->p_v, h->p_diag, h->st));
  // symmetric pattern is required by the level construction and IC(0)
  TRY_CUDA(cudaMemsetAsync(h->flag, 0, sizeof(int), h->st));
  TRY_CUDA(mirror_map(N, h->p_rp, h->p_ci, h->p_diag, h->mir, h->flag, h->st));
  int bad = 0;
  TRY(to_host(h, &bad, h->flag, 1));
  TRY(sync(h, "mirror map"));
  if (bad) return fail(SDSL_ERR_ARG, "the system matrix must have a symmetric sparsity pattern");
  // level sets (lower and upper) of the block triangular solves
  int32_t *cnt, *fa, *fb, *nlev_d;
  Arena tmp;
  tmp.st = h->st;
  tmp.track(&h->live_bytes, &h->peak_bytes);
  TRY(tmp.get(&cnt, N));
  TRY(h->pc.get(&h->row_lev_lo, N));
  TRY(h->pc.get(&h->row_lev_up, N));
  TRY(tmp.get(&fa, N));
  TRY(tmp.get(&fb, N));
  TRY(tmp.get(&nlev_d, nb));
  TRY(build_levels(h, 0, &h->lev_off_lo, &h->lev_ptr_lo, &h->lev_rows_lo, h->h_nlev_lo, &h->tot_lo, cnt,
                   h->row_lev_lo, fa, fb, nlev_d));
  TRY(build_levels(h, 1, &h->lev_off_up, &h->lev_ptr_up, &h->lev_rows_up, h->h_nlev_up, &h->tot_up, cnt,
                   h->row_lev_up, fa, fb, nlev_d));
  // per-block factorization with the shift-retry rule: a block is factored
  // with diagonal p_ii + alpha p_ii for the first alpha of the ladder whose
  // factor does not break down
  static const double kShifts[5] = {0.0, 1e-3, 1e-2, 1e-1, 1.0};
  constexpr int kNS = 5;
  std::vector<int> tries(nb, 0);
  h->h_alpha.assign(nb, 0.0);
  int64_t shifted = 0;
  if (bj_method(h)) {
    // IC(0): every shift of the ladder at once (nblocks x 5 CTAs), then pick
    double *Fall, *dinv_all, *d_alpha;
    int32_t *d_status, *d_choice;
    TRY(tmp.get(&Fall, (size_t)kNS * h->p_nnz));
    TRY(tmp.get(&dinv_all, (size_t)kNS * N));
    TRY(h->pc.get(&d_alpha, kNS));
    TRY(h->pc.get(&d_status, nb * kNS));
    TRY(h->pc.get(&d_choice, nb));
    TRY(to_dev(h, d_alpha, kShifts, kNS));
    // largest blocks first: their factorizations start in the first wave
    std::vector<int32_t> order(nb);
    for (int64_t k = 0; k < nb; ++k) order[k] = (int32_t)k;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return h->h_bp[a + 1] - h->h_bp[a] > h->h_bp[b + 1] - h->h_bp[b];
    });
    int32_t* d_order;
    TRY(h->pc.get(&d_order, nb));
    TRY(to_dev(h, d_order, order.data(), nb));
    TRY_CUDA(ic0_factor_all(nb, h->d_bp, h->p_rp, h->p_ci, h->p_v, h->p_diag, h->lev_off_lo, h->lev_ptr_lo,
                            h->lev_rows_lo, d_alpha, kNS, h->p_nnz, N, Fall, dinv_all, d_status, d_order, h->st));
    std::vector<int32_t> status(nb * kNS), choice(nb);
    TRY(to_host(h, status.data(), d_status, nb * kNS));
    TRY(sync(h, "factor"));
    for (int64_t k = 0; k < nb; ++k) {
      int t = 0;
      while (t < kNS && status[k * kNS + t]) ++t;
      if (t == kNS) {
        h->h_alpha[k] = -1.0;
        tmp.release();
        return fail(SDSL_ERR_BREAKDOWN, "block " + std::to_string(k) + " breaks down with every diagonal shift");
      }
      choice[k] = t;
      tries[k] = t;
    }
    TRY(to_dev(h, d_choice, choice.data(), nb));
    TRY_CUDA(pick_shift(h->d_bp, h->p_rp, d_choice, h->p_nnz, N, Fall, dinv_all, h->F, h->dinv, h->row_block,
                        h->h_bp[nb], h->st));
    tmp.release();
  } else {
    double* d_alpha;
    int32_t *d_active, *d_status;
    TRY(h->pc.get(&d_alpha, nb));
    TRY(h->pc.get(&d_active, nb));
    TRY(h->pc.get(&d_status, nb));
    std::vector<int32_t> active(nb, 1), status(nb, 0);
    for (int round = 0; round < kNS; ++round) {
      for (int64_t k = 0; k < nb; ++k) h->h_alpha[k] = kShifts[tries[k]];
      TRY(to_dev(h, d_alpha, h->h_alpha.data(), nb));
      TRY(to_dev(h, d_active, active.data(), nb));
      TRY_CUDA(ilu0_factor(nb, h->d_bp, h->p_rp, h->p_ci, h->p_v, h->p_diag, h->lev_off_lo, h->lev_ptr_lo,
                           h->lev_rows_lo, d_alpha, d_active, h->F, h->dinv, d_status, h->st));
      TRY(to_host(h, status.data(), d_status, nb));
      TRY(sync(h, "factor"));
      bool any = false;
      for (int64_t k = 0; k < nb; ++k) {
        if (active[k] && status[k]) {
          any = true;
          if (++tries[k] >= kNS) {
            h->h_alpha[k] = -1.0;
            return fail(SDSL_ERR_BREAKDOWN, "block " + std::to_string(k) + " breaks down with every diagonal shift");
          }
        } else {
          active[k] = 0;
        }
      }
      if (!any) break;
    }
  }
  tmp.release();
  for (int64_t k = 0; k < nb; ++k) {
    h->h_alpha[k] = kShifts[tries[k]];
    shifted += tries[k] > 0;
  }
  const bool b16 = h->opt.factor_prec == 16;  // BF16 storage (staged solves): FP32 arrays hold the rounded values
  const bool f32 = h->opt.factor_prec == 32 || b16;
  if (f32) {
    TRY(h->pc.get(&h->Ff, h->p_nnz));
    TRY(h->pc.get(&h->dinvf, N));
  } else {
    h->Ff = nullptr;
    h->dinvf = nullptr;
  }
  if (bbd_method(h->method)) {
    if (f32) {
      TRY_CUDA(to_float(h->p_nnz, h->F, h->Ff, h->st));
      TRY_CUDA(to_float(N, h->dinv, h->dinvf, h->st));
    }
  } else {
    TRY_CUDA(ic0_finish(N, h->p_nnz, h->p_rp, h->p_diag, h->mir, h->F, h->dinv, h->Ff, h->dinvf, h->st));
    if (b16) {
      TRY_CUDA(round_bf16(h->p_nnz, h->Ff, h->st));
      TRY_CUDA(round_bf16(N, h->dinvf, h->st));
    }
  }
  if (bbd_method(h->method)) {
    TRY(build_bbd(h));
    const int mres = std::max(1, h->opt.restart);
    TRY(h->pc.get(&h->V, (size_t)(mres + 1) * N));
    TRY(h->pc.get(&h->Z, (size_t)mres * N));
    TRY(h->pc.get(&h->gpart, (size_t)(mres + 1) * multidot_grid(N)));
    TRY(h->pc.get(&h->gh, 2 * (mres + 1) + 2));
  }
  // apply plan
  int64_t maxb = 0;
  for (int64_t k = 0; k < nb; ++k) maxb = std::max(maxb, h->h_bp[k + 1] - h->h_bp[k]);
  TriSolve& M = h->M;
  M = TriSolve{};
  M.nblocks = nb;
  M.bp = h->d_bp;
  M.prp = h->p_rp;
  M.pci = h->p_ci;
  M.pdiag = h->p_diag;
  M.F = h->F;
  M.Ff = h->Ff;
  M.dinv = h->dinv;
  M.dinvf = h->dinvf;
  M.lev_off_lo = h->lev_off_lo;
  M.lev_ptr_lo = h->lev_ptr_lo;
  M.lev_rows_lo = h->lev_rows_lo;
  M.lev_off_up = h->lev_off_up;
  M.lev_ptr_up = h->lev_ptr_up;
  M.lev_rows_up = h->lev_rows_up;
  M.unit_lower = bbd_method(h->method) ? 1 : 0;
  M.prec = b16 ? 16 : f32 ? 32 : 64;
  const double avg_half = N > 0 ? (double)(h->p_nnz - N) / (2.0 * (double)N) : 1.0;
  M.lanes = pow2_lanes(avg_half, 2.0);
  M.max_block = maxb;
  if ((size_t)maxb * (f32 ? 4 : 8) > (size_t)200 * 1024) {
    if (f32) TRY(h->pc.get(&M.yscratch, N));
    else TRY(h->pc.get(&M.yscratch64, N));
  }
  TRY(h->pc.get(&h->part_blk, 3 * nb + 32));
  // level-ordered packed triangles for the flag-synchronised solves
  // Auto: FP32-stored factors are applied in float-float arithmetic (48) by
  // the staged sweeps -- one fixed linear operator to ~1e-14, as both PCG and
  // BiCGSTAB assume, on the FP32 pipes; the other solve kernels apply them in
  // FP64 arithmetic.  An FP32-arithmetic apply (32) is linear only to ~1e-7;
  // PCG then needs the flexible beta.
  int apply = h->opt.apply_prec != 0 ? h->opt.apply_prec : f32 ? 48 : 64;
  if (!f32) apply = 64;
  M.apply_prec = apply;
  M.threads = 1024;
  const bool fits = sf_smem_bytes(maxb, apply == 32 ? 4 : 8) <= (size_t)200 * 1024;
  M.slot_bytes = apply == 32 ? 1536 : 1024;
  const double avg_half2 = N > 0 ? (double)(h->p_nnz - N) / (2.0 * (double)N) : 1.0;
  const int sweep_lanes = std::max(4, pow2_lanes(avg_half2, 4.0));
  // bound of the staged tile offsets: every level padded to whole tiles of
  // RW rows -> at most rows/RW + levels tiles per direction
  {
    const int64_t RWb = 32 / sweep_lanes;
    int64_t mt = 0;
    for (int64_t k = 0; k < nb; ++k) {
      const int64_t rows = h->h_bp[k + 1] - h->h_bp[k];
      mt = std::max<int64_t>(mt, 2 * (rows / RWb + 1) + h->h_nlev_lo[k] + h->h_nlev_up[k]);
    }
    M.max_tiles = mt;
  }
  const bool fits_staged = staged_smem_bytes(maxb, apply == 32 ? 4 : 8, 16, 1024, 2, M.max_tiles, 0) <= (size_t)225 * 1024;
  if ((h->opt.solve_kernel == 2 && !fits) || (h->opt.solve_kernel == 3 && !fits_staged))
    return fail(SDSL_ERR_ARG, "flag-synchronised solves need the largest block to fit in shared memory");
  M.staged = (bj_method(h) && (h->opt.solve_kernel == 3 || (h->opt.solve_kernel == 0 && fits_staged))) ? 1 : 0;
  M.sweep_warps = h->opt.sweep_warps > 0 ? h->opt.sweep_warps : 16;
  M.backoff_ns = h->opt.sweep_backoff_ns >= 0 ? h->opt.sweep_backoff_ns : 0;
  M.wait_limit = h->opt.wait_limit > 0 ? h->opt.wait_limit : h->opt.wait_test ? 1024 : (1 << 23);
  M.wait_pad = h->opt.wait_test ? 1 : 0;
  if (M.staged) {
    bool ok = false;
    int E = h->opt.sweep_lane_entries > 0 ? h->opt.sweep_lane_entries : 16;
    int gap = h->opt.sweep_wait == 3 ? 1 : h->opt.sweep_far_gap > 0 ? h->opt.sweep_far_gap : 3;
    if (h->opt.tune) {
      const TuneKey key = tune_key(h, apply);
      TuneChoice ch{};
      {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = tune_cache().find(key);
        if (it != tune_cache().end()) ch = it->second;
      }
      if (ch.E == 0) {
        auto t0 = std::chrono::steady_clock::now();
        TRY(tune_sweep(h, f32, apply, &ch.E, &ch.gap));
        ch.ms += std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
        h->stats.ms_tune += ch.ms;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        TuneChoice& c = tune_cache()[key];
        c.E = ch.E;
        c.gap = ch.gap;
      }
      E = ch.E;
      gap = ch.gap;
    }
    h->stats.sweep_shape[0] = E;
    h->stats.sweep_shape[1] = gap;
    TRY(build_vtiles(h, f32, apply, E, gap, h->pc, &ok));
    if (!ok) {
      if (h->opt.solve_kernel == 3)
        return fail(SDSL_ERR_ARG, "staged solves need blocks of at most 65,535 rows that fit in shared memory");
      M.staged = 0;
    }
  }
  if (b16 && !M.staged)
    return fail(SDSL_ERR_ARG, "BF16 factors (factor_prec 16) need the staged solves (blocks of at most 65,535 rows "
                              "that fit in shared memory)");
  // float-float arithmetic exists in the staged sweeps only
  if (M.apply_prec == 48 && !M.staged) {
    if (h->opt.apply_prec == 48)
      return fail(SDSL_ERR_ARG, "the float-float apply (apply_prec 48) needs the staged solves (solve_kernel 0 or 3)");
    M.apply_prec = 64;
  }
  M.flexible = h->opt.flexible < 0 ? (M.apply_prec == 32 ? 1 : 0) : (h->opt.flexible ? 1 : 0);
  M.sync_free = (bj_method(h) && !M.staged && (h->opt.solve_kernel == 2 || (h->opt.solve_kernel == 0 && fits)))
                    ? 1 : 0;
  if (M.sync_free) {
    M.lanes = sweep_lanes;
    const int RW = 32 / M.lanes;
    const int64_t nrows = h->h_bp[nb];
    const size_t vs = f32 ? 4 : 8;
    std::vector<int32_t> lptr, lrows, sched;
    std::vector<int64_t> pos(nb + 1);
    for (int dir = 0; dir < 2; ++dir) {
      const int64_t tot = dir == 0 ? h->tot_lo : h->tot_up;
      const std::vector<int32_t>& nl = dir == 0 ? h->h_nlev_lo : h->h_nlev_up;
      lptr.resize(tot + 1);
      lrows.resize(nrows);
      TRY(to_host(h, lptr.data(), dir == 0 ? h->lev_ptr_lo : h->lev_ptr_up, tot + 1));
      TRY(to_host(h, lrows.data(), dir == 0 ? h->lev_rows_lo : h->lev_rows_up, nrows));
      TRY(sync(h, "schedule"));
      // rows in level order, every level padded to whole warp tiles (-1)
      sched.clear();
      int64_t L = 0;
      for (int64_t k = 0; k < nb; ++k) {
        pos[k] = (int64_t)sched.size();
        for (int32_t l = 0; l < nl[k]; ++l, ++L) {
          for (int32_t q = lptr[L]; q < lptr[L + 1]; ++q) sched.push_back(lrows[q]);
          while (sched.size() % RW) sched.push_back(-1);
        }
      }
      pos[nb] = (int64_t)sched.size();
      const int64_t npos = pos[nb];
      int32_t *d_sched, *col, *prow;
      int64_t *off, *d_pos;
      void *val, *pdv;
      TRY(h->pc.get(&d_sched, npos));
      TRY(h->pc.get(&d_pos, nb + 1));
      TRY(to_dev(h, d_sched, sched.data(), npos));
      TRY(to_dev(h, d_pos, pos.data(), nb + 1));
      TRY(h->pc.get(&off, npos + 1));
      TRY_CUDA(pack_count(dir, npos, h->row_block, h->d_bp, h->p_rp, h->p_ci, h->p_diag, d_sched, off, h->st));
      int64_t tot_e = 0;
      TRY(scan_total(h, off, npos, &tot_e));
      TRY(h->pc.get(&col, tot_e));
      TRY(h->pc.get(reinterpret_cast<unsigned char**>(&val), tot_e * vs));
      TRY(h->pc.get(reinterpret_cast<unsigned char**>(&pdv), npos * vs));
      TRY(h->pc.get(&prow, npos));
      TRY_CUDA(pack_fill(dir, npos, h->row_block, h->d_bp, h->p_rp, h->p_ci, h->p_diag, d_sched, h->F, h->dinv,
                         f32 ? 32 : 64, off, col, val, pdv, prow, h->st));
      if (dir == 0) { M.fwd_off = off; M.fwd_col = col; M.fwd_val = val; M.fwd_dinv = pdv; M.fwd_row = prow; M.fwd_pos = d_pos; }
      else { M.bwd_off = off; M.bwd_col = col; M.bwd_val = val; M.bwd_dinv = pdv; M.bwd_row = prow; M.bwd_pos = d_pos; }
    }
  }
  TRY(plan_long_rows(h));
  TRY(plan_sell(h));
  choose_spmv_plan(h);
  if (h->opt.tune) TRY(tune_spmv(h));
  if (bj_method(h) && !h->opt.profile) TRY(build_graph(h));
  cudaEventRecord(h->ev_b, h->st);
  TRY(sync(h, "factor end"));
  h->factored = true;
  h->need_rebuild = false;
  h->iters_post_build = -1;
  h->solves_since_build = 0;
  h->tau_built = tau;
  h->stats.tau_used = tau;
  h->stats.ms_factor = elapsed(h);
  h->stats.nnz_precond = h->p_nnz;
  h->stats.nnz_factor = bbd_method(h->method) ? h->p_nnz : (h->p_nnz + N) / 2;
  h->stats.spmv_lanes = h->A.lanes;
  h->stats.product_lanes[0] = h->A.factored ? (h->A.sell ? -1 : h->A.at_lanes) : 0;
  h->stats.product_lanes[1] = h->A.factored ? (h->A.sell ? -1 : h->A.a_lanes) : 0;
  h->stats.solve_lanes = h->M.lanes;
  h->stats.levels_lower = h->tot_lo;
  h->stats.levels_upper = h->tot_up;
  int64_t mx = 0;
  for (int64_t k = 0; k < nb; ++k) mx = std::max<int64_t>(mx, std::max(h->h_nlev_lo[k], h->h_nlev_up[k]));
  h->stats.max_levels = mx;
  h->stats.shifted_blocks = shifted;
  h->stats.builds += 1;
  // Algorithmic HBM bytes per launch of the three PCG kernels: every array
  // the kernel must touch, once (gathers of vector entries counted once).
  //  SpMV:    values + columns of S (12 B/nnz), row pointers, read p, write q.
  //  update:  read p, q, x, r; write x, r, z; strict lower and upper factor
  //           values + columns; inverse diagonal; row pointers and diagonal
  //           positions (read by both solves); level row lists (both solves).
  //  direct.: read z, p; write p.
  const double sf = b16 ? 2.0 : f32 ? 4.0 : 8.0;
  const double Nd = (double)N;
  const double offd = (double)(h->p_nnz - N);
  h->stats.kernel_bytes[0] = 12.0 * (double)h->s_nnz + 8.0 * (Nd + 1.0) + 16.0 * Nd;
  if (h->A.factored)  // A^T p (+theta, u) then A u (+p, q): both CSR streams once
    h->stats.kernel_bytes[0] = 24.0 * (double)h->a_nnz + 8.0 * ((double)h->n + 1.0) + 8.0 * (Nd + 1.0) +
                               8.0 * Nd + 24.0 * (double)h->n + 16.0 * Nd;
  h->stats.kernel_bytes[1] = 56.0 * Nd + (sf + 4.0) * offd + sf * Nd + 2.0 * 8.0 * (Nd + 1.0) + 2.0 * 8.0 * Nd +
                             2.0 * 4.0 * Nd;
  h->stats.kernel_bytes[2] = 24.0 * Nd;
  h->stats.kernel_bytes[3] = 0.0;
  h->stats.bytes_per_iter = h->stats.kernel_bytes[0] + h->stats.kernel_bytes[1] + h->stats.kernel_bytes[2];
  return SDSL_OK;
}

sdsl_status pcg_solve(sdsl_handle h, sdsl_stats* st_out) {
  const int64_t N = h->N;
  // ||b||^2 and r = b - S x
  double* bn2 = h->scalars;
  TRY_CUDA(norm2_sq(N, h->b, h->part, bn2, reinterpret_cast<unsigned int*>(h->part + 152 * 32), h->st));
  TRY_CUDA(pcg_init_state(h->state, 0.0, h->opt.maxit, h->st));
  TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 1, h->st));
  double bnorm2 = 0.0;
  TRY(to_host(h, &bnorm2, bn2, 1));
  TRY(to_host(h, h->h_state, h->state, 1));
  TRY(sync(h, "pcg init"));
  const double tol = h->opt.rtol * std::sqrt(bnorm2);
  const double tol2 = tol * tol;
  sdsl_stats& S = h->stats;
  S.iters = 0;
  S.restarts = 0;
  if (bnorm2 == 0.0) {
    TRY_CUDA(cudaMemsetAsync(h->x, 0, sizeof(double) * (size_t)N, h->st));
    S.rel_res_true = S.rel_res_rec = 0.0;
    S.status = SDSL_OK;
    return SDSL_OK;
  }
  if (h->h_state->tr <= tol2) {
    S.rel_res_true = S.rel_res_rec = std::sqrt(h->h_state->tr / bnorm2);
    S.status = SDSL_OK;
    return SDSL_OK;
  }
  TRY_CUDA(pcg_init_state(h->state, tol2, h->opt.maxit, h->st));
  TRY_CUDA(precond_apply(h->M, h->r, h->z, h->p, h->part_blk, h->state, 1, h->st));
  sdsl_status result = SDSL_ERR_NOT_CONVERGED;
  for (;;) {
    if (h->opt.profile) {
      TRY(profiled_iteration(h));
    } else if (h->graph) {
      TRY_CUDA(cudaGraphLaunch(h->graph, h->st));
      count_launch(h->graph_kernels);
    } else {
      for (int i = 0; i < 8; ++i) TRY(enqueue_pcg_iteration(h));
    }
    TRY(to_host(h, h->h_state, h->state, 1));
    TRY(sync(h, "pcg iterations"));
    const PcgState& hs = *h->h_state;
    if (hs.err) return fail(SDSL_ERR_TIMEOUT, "a triangular-solve wait exceeded its bound");
    if (!hs.done) continue;
    if (hs.done == 3) { result = SDSL_ERR_BREAKDOWN; break; }
    if (hs.done == 2) { result = SDSL_ERR_NOT_CONVERGED; break; }
    // recurrence converged: confirm with the true residual
    TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 0, h->st));
    TRY(to_host(h, h->h_state, h->state, 1));
    TRY(sync(h, "true residual"));
    if (h->h_state->tr <= tol2) { result = SDSL_OK; break; }
    if (h->h_state->iters >= h->opt.maxit) { result = SDSL_ERR_NOT_CONVERGED; break; }
    // restart from r = b - S x with a fresh direction
    S.restarts += 1;
    TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 1, h->st));
    TRY_CUDA(precond_apply(h->M, h->r, h->z, h->p, h->part_blk, h->state, 1, h->st));
    TRY_CUDA(cudaMemsetAsync(&h->state->done, 0, sizeof(int), h->st));
  }
  // final true residual (also for not-converged / breakdown exits)
  TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 0, h->st));
  TRY(to_host(h, h->h_state, h->state, 1));
  TRY(sync(h, "final residual"));
  S.iters = h->h_state->iters;
  S.rel_res_true = std::sqrt(h->h_state->tr / bnorm2);
  S.rel_res_rec = std::sqrt(h->h_state->rr / bnorm2);
  S.status = result;
  (void)st_out;
  if (result == SDSL_OK) return SDSL_OK;
  return fail(result, result == SDSL_ERR_BREAKDOWN ? "PCG breakdown (p^T S p <= 0 or non-finite)"
                                                   : "PCG reached maxit before the tolerance");
}

// ------------------------------------------------------------- batched PCG
// Several Block-Jacobi PCG solves (independent requests, each its own handle)
// advanced together: every iteration is three persistent launches over a
// device table of (request, virtual CTA) items -- the factored product on
// the sliced ELL copies, the update with the staged block sweeps, the
// direction -- so one launch carries the blocks of every request; each
// request keeps its own grids, partial sums, tickets and scalars, so its
// arithmetic is that of its solve alone.  Iterations are captured G at a
// time in one CUDA graph; after each graph launch the host reads every
// request's state and, as pcg_solve does for one, confirms a converged
// recurrence with the true residual or restarts it.  Requests that stopped
// are skipped by the kernels.
bool batchable(const sdsl_handle h, const sdsl_handle h0) {
  const TriSolve& M = h->M;
  const TriSolve& M0 = h0->M;
  return h->method == SDSL_BJ_PCG && h->factored && M.staged && h->A.factored && h->A.sell && h->dev == h0->dev &&
         M.prec == M0.prec && M.apply_prec == M0.apply_prec && M.slots == M0.slots && M.kreg == M0.kreg &&
         !h->opt.profile;
}

struct BatchTrack {
  double bnorm2 = 0.0, tol2 = 0.0;
  int state = 0;  // 0 running, 1 finished
  sdsl_status result = SDSL_ERR_NOT_CONVERGED;
};

}  // namespace

// A continuous batch: requests join (sdsl_batch_add) and leave (when their
// solve ends, reported by sdsl_batch_step) between graph launches.
struct sdsl_batch_s {
  struct Member {
    sdsl_handle h;
    const double* b;
    double* x;
    int x0_zero, rebuilt;
    bool reused;
    BatchTrack tr;
    cudaEvent_t t0;  // when the member joined (its solve time runs from there)
  };
  int dev = 0, sms = 152;
  cudaStream_t st = nullptr;
  std::vector<Member> members;
  Arena ar;
  cudaGraphExec_t graph = nullptr;
  long long graph_kernels = 0;
  bool dirty = true;
  int graph_iters = 16;
  // the launch tables of the current members
  BatchReq* d_reqs = nullptr;
  BatchItem *d_at = nullptr, *d_a = nullptr, *d_up = nullptr, *d_dir = nullptr;
  int n_at = 0, n_a = 0, n_up = 0, n_dir = 0;
  size_t smem = 0;
  TriSolve M0{};
};

namespace {

// Begin a member's solve on the batch stream (the first part of pcg_solve):
// ||b||, r = b - S x, and -- unless the tolerance is met already -- z, p, rho.
sdsl_status batch_begin(sdsl_batch B, sdsl_batch_s::Member& mb) {
  sdsl_handle h = mb.h;
  const cudaStream_t bs = B->st;
  double* bn2 = h->scalars;
  TRY_CUDA(norm2_sq(h->N, h->b, h->part, bn2, reinterpret_cast<unsigned int*>(h->part + 152 * 32), bs));
  TRY_CUDA(pcg_init_state(h->state, 0.0, h->opt.maxit, bs));
  TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 1, bs));
  double bn = 0.0;
  TRY_CUDA(cudaMemcpyAsync(&bn, bn2, sizeof(double), cudaMemcpyDeviceToHost, bs));
  TRY_CUDA(cudaMemcpyAsync(h->h_state, h->state, sizeof(PcgState), cudaMemcpyDeviceToHost, bs));
  TRY_CUDA(cudaStreamSynchronize(bs));
  h->stats.iters = 0;
  h->stats.restarts = 0;
  mb.tr.bnorm2 = bn;
  const double tol = h->opt.rtol * std::sqrt(bn);
  mb.tr.tol2 = tol * tol;
  static const int kDone = 1;  // a finished member never runs in the kernels
  if (bn == 0.0 || h->h_state->tr <= mb.tr.tol2) {
    if (bn == 0.0) TRY_CUDA(cudaMemsetAsync(h->x, 0, sizeof(double) * (size_t)h->N, bs));
    TRY_CUDA(cudaMemcpyAsync(&h->state->done, &kDone, sizeof(int), cudaMemcpyHostToDevice, bs));
    mb.tr.state = 1;
    mb.tr.result = SDSL_OK;
    return SDSL_OK;
  }
  TRY_CUDA(pcg_init_state(h->state, mb.tr.tol2, h->opt.maxit, bs));
  TRY_CUDA(precond_apply(h->M, h->r, h->z, h->p, h->part_blk, h->state, 1, bs));
  return SDSL_OK;
}

// One batched PCG iteration over the current tables (three launches).
cudaError_t batch_iteration(sdsl_batch B) {
  SDSL_CUDA_TRY(batch_product(B->d_reqs, B->d_at, B->n_at, B->d_a, B->n_a, B->sms * 8, B->st));
  SDSL_CUDA_TRY(batch_update(B->M0, B->d_reqs, B->d_up, B->n_up, B->sms, B->smem, B->st));
  return batch_direction(B->d_reqs, B->d_dir, B->n_dir, B->sms * 8, B->st);
}

// The launch tables and graph of the running members.
sdsl_status batch_plan(sdsl_batch B) {
  if (B->graph) { cudaGraphExecDestroy(B->graph); B->graph = nullptr; }
  B->ar.release();
  std::vector<BatchReq> reqs;
  std::vector<BatchItem> it_at, it_a, it_up, it_dir;
  std::vector<std::pair<int64_t, BatchItem>> blocks;
  B->smem = 0;
  for (auto& mb : B->members) {
    if (mb.tr.state != 0) continue;
    sdsl_handle h = mb.h;
    const int i = (int)reqs.size();
    BatchReq R{};
    R.M = h->M;
    R.A = h->A;
    R.x = h->x; R.r = h->r; R.z = h->z; R.p = h->p; R.q = h->q;
    R.part = h->part;
    R.part_blk = h->part_blk;
    R.s = h->state;
    R.n = h->N;
    R.g_at = (int)h->A.sell_at_grid;
    R.g_a = (int)h->A.sell_a_grid;
    R.g_dir = direction_grid(h->N);
    reqs.push_back(R);
    for (int v = 0; v < R.g_at; ++v) it_at.push_back(BatchItem{i, v});
    for (int v = 0; v < R.g_a; ++v) it_a.push_back(BatchItem{i, v});
    for (int v = 0; v < R.g_dir; ++v) it_dir.push_back(BatchItem{i, v});
    for (int64_t k = 0; k < h->nblocks; ++k)
      blocks.emplace_back(h->h_bp[k + 1] - h->h_bp[k], BatchItem{i, (int32_t)k});
    B->smem = std::max(B->smem, staged_smem_bytes_of(h->M));
    B->M0 = h->M;
  }
  B->dirty = false;
  B->n_at = (int)it_at.size();
  B->n_a = (int)it_a.size();
  B->n_dir = (int)it_dir.size();
  B->n_up = (int)blocks.size();
  if (reqs.empty()) return SDSL_OK;
  // blocks of the update: largest first over all members (longest work starts first)
  std::stable_sort(blocks.begin(), blocks.end(),
                   [](const std::pair<int64_t, BatchItem>& x, const std::pair<int64_t, BatchItem>& y) {
                     return x.first > y.first;
                   });
  for (auto& e : blocks) it_up.push_back(e.second);
  const cudaStream_t bs = B->st;
  TRY(B->ar.get(&B->d_reqs, reqs.size()));
  TRY(B->ar.get(&B->d_at, it_at.size()));
  TRY(B->ar.get(&B->d_a, it_a.size()));
  TRY(B->ar.get(&B->d_up, it_up.size()));
  TRY(B->ar.get(&B->d_dir, it_dir.size()));
  TRY_CUDA(cudaMemcpyAsync(B->d_reqs, reqs.data(), sizeof(BatchReq) * reqs.size(), cudaMemcpyHostToDevice, bs));
  TRY_CUDA(cudaMemcpyAsync(B->d_at, it_at.data(), sizeof(BatchItem) * it_at.size(), cudaMemcpyHostToDevice, bs));
  TRY_CUDA(cudaMemcpyAsync(B->d_a, it_a.data(), sizeof(BatchItem) * it_a.size(), cudaMemcpyHostToDevice, bs));
  TRY_CUDA(cudaMemcpyAsync(B->d_up, it_up.data(), sizeof(BatchItem) * it_up.size(), cudaMemcpyHostToDevice, bs));
  TRY_CUDA(cudaMemcpyAsync(B->d_dir, it_dir.data(), sizeof(BatchItem) * it_dir.size(), cudaMemcpyHostToDevice, bs));
  if (B->graph_iters <= 0) return SDSL_OK;
  cudaGraph_t g = nullptr;
  const long long before = launches_so_far();
  TRY_CUDA(cudaStreamBeginCapture(bs, cudaStreamCaptureModeRelaxed));
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < B->graph_iters && e == cudaSuccess; ++k) e = batch_iteration(B);
  cudaError_t e2 = cudaStreamEndCapture(bs, &g);
  B->graph_kernels = launches_so_far() - before;
  count_launch(-B->graph_kernels);  // captured, not executed: counted per graph launch
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e != cudaSuccess ? e : e2, "batched iteration capture");
  }
  e = cudaGraphInstantiate(&B->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate (batch)");
  return SDSL_OK;
}

// Right-preconditioned BiCGSTAB with the Block-Jacobi IC(0) preconditioner
// (Sec. 4.3 pairs them).  The count is the number of passes started; a pass
// whose first half already meets the tolerance ends there.  Convergence of
// the recurrence is confirmed with the true residual; if that is still above
// the tolerance the iteration restarts from r = b - S x (new shadow vector).
sdsl_status bicg_solve(sdsl_handle h) {
  const int64_t N = h->N;
  double* bn2 = h->scalars;
  TRY_CUDA(norm2_sq(N, h->b, h->part, bn2, reinterpret_cast<unsigned int*>(h->part + 152 * 32), h->st));
  TRY_CUDA(pcg_init_state(h->state, 0.0, h->opt.maxit, h->st));
  TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 1, h->st));
  double bnorm2 = 0.0;
  TRY(to_host(h, &bnorm2, bn2, 1));
  TRY(to_host(h, h->h_state, h->state, 1));
  TRY(sync(h, "bicgstab init"));
  const double tol = h->opt.rtol * std::sqrt(bnorm2);
  const double tol2 = tol * tol;
  sdsl_stats& S = h->stats;
  S.iters = 0;
  S.restarts = 0;
  if (bnorm2 == 0.0) {
    TRY_CUDA(cudaMemsetAsync(h->x, 0, sizeof(double) * (size_t)N, h->st));
    S.rel_res_true = S.rel_res_rec = 0.0;
    S.status = SDSL_OK;
    return SDSL_OK;
  }
  S.rel_res_true = S.rel_res_rec = std::sqrt(h->h_state->tr / bnorm2);
  if (h->h_state->tr <= tol2) {
    S.status = SDSL_OK;
    return SDSL_OK;
  }
  if (h->opt.maxit == 0) {
    S.status = SDSL_ERR_NOT_CONVERGED;
    return fail(SDSL_ERR_NOT_CONVERGED, "BiCGSTAB reached maxit before the tolerance");
  }
  // the pass limit is tested by k_bicg_finish; the mode-0 update's own limit
  // test is kept out of the way
  const long long kNoLimit = (long long)1 << 62;
  TRY_CUDA(pcg_init_state(h->state, tol2, kNoLimit, h->st));
  TRY_CUDA(bicg_init(h->bicg, h->opt.maxit, h->st));
  TRY_CUDA(bicg_restart(N, h->r, h->rt, h->bicg, h->st));
  sdsl_status result = SDSL_ERR_NOT_CONVERGED;
  for (;;) {
    if (h->graph) {
      TRY_CUDA(cudaGraphLaunch(h->graph, h->st));
      count_launch(h->graph_kernels);
    } else {
      for (int i = 0; i < 4; ++i) TRY(enqueue_bicg_iteration(h));
    }
    TRY(to_host(h, h->h_state, h->state, 1));
    TRY(sync(h, "bicgstab passes"));
    const PcgState& hs = *h->h_state;
    if (hs.err) return fail(SDSL_ERR_TIMEOUT, "a triangular-solve wait exceeded its bound");
    if (!hs.done) continue;
    if (hs.done == 3) { result = SDSL_ERR_BREAKDOWN; break; }
    if (hs.done == 2) { result = SDSL_ERR_NOT_CONVERGED; break; }
    TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 0, h->st));
    TRY(to_host(h, h->h_state, h->state, 1));
    TRY(sync(h, "true residual"));
    if (h->h_state->tr <= tol2) { result = SDSL_OK; break; }
    if (h->h_state->iters >= h->opt.maxit) { result = SDSL_ERR_NOT_CONVERGED; break; }
    S.restarts += 1;
    TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 1, h->st));
    TRY_CUDA(bicg_restart(N, h->r, h->rt, h->bicg, h->st));
    TRY_CUDA(cudaMemsetAsync(&h->state->done, 0, sizeof(int), h->st));
  }
  TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 0, h->st));
  TRY(to_host(h, h->h_state, h->state, 1));
  TRY(sync(h, "final residual"));
  S.iters = h->h_state->iters;
  S.rel_res_true = std::sqrt(h->h_state->tr / bnorm2);
  S.rel_res_rec = std::sqrt(h->h_state->rr / bnorm2);
  S.status = result;
  if (result == SDSL_OK) return SDSL_OK;
  return fail(result, result == SDSL_ERR_BREAKDOWN ? "BiCGSTAB breakdown (a zero or non-finite scalar)"
                                                   : "BiCGSTAB reached maxit before the tolerance");
}

}  // namespace

// ------------------------------------------------------------- one solve
// The pieces of sdsl_solve (also used by sdsl_batch_solve for every request).

// Rebuild if the reuse rule asked for it; copy b and the initial guess.
sdsl_status solve_prepare(sdsl_handle h, const double* b, const double* x, int x0_zero, int* rebuilt) {
  *rebuilt = 0;
  if (h->need_rebuild) {
    TRY(factor_impl(h));
    *rebuilt = 1;
  }
  TRY(to_dev(h, h->b, b, h->N));
  if (!x0_zero) TRY(to_dev(h, h->x0, x, h->N));
  if (x0_zero) TRY_CUDA(cudaMemsetAsync(h->x, 0, sizeof(double) * (size_t)h->N, h->st));
  else TRY_CUDA(cudaMemcpyAsync(h->x, h->x0, sizeof(double) * (size_t)h->N, cudaMemcpyDeviceToDevice, h->st));
  return SDSL_OK;
}

// One Krylov solve from the initial guess (x0 or zero); ms_solve is its
// device time.
sdsl_status solve_attempt(sdsl_handle h, int x0_zero, sdsl_stats* st) {
  cudaEventRecord(h->ev_a, h->st);
  if (x0_zero) TRY_CUDA(cudaMemsetAsync(h->x, 0, sizeof(double) * (size_t)h->N, h->st));
  else TRY_CUDA(cudaMemcpyAsync(h->x, h->x0, sizeof(double) * (size_t)h->N, cudaMemcpyDeviceToDevice, h->st));
  sdsl_status s = h->method == SDSL_BBD_GMRES      ? gmres_solve(h)
                  : h->method == SDSL_BBD_GCR     ? gcr_solve(h)
                  : h->method == SDSL_BJ_BICGSTAB ? bicg_solve(h)
                                                  : pcg_solve(h, st);
  cudaEventRecord(h->ev_b, h->st);
  sdsl_status e = sync(h, "solve end");
  if (e != SDSL_OK) return e;
  h->stats.ms_solve = elapsed(h);
  return s;
}

// After the first attempt (status s): the reuse rule's and the filter
// relaxation's repeated solves, the copy-out of x, the statistics and the
// reuse bookkeeping for the next solve.
sdsl_status solve_conclude(sdsl_handle h, double* x, int x0_zero, sdsl_stats* st, sdsl_status s, bool reused,
                           int rebuilt) {
  int64_t discarded = 0;
  // Reuse rule (Sec. 3.4), failure branch: a reused preconditioner under
  // which the solve did not converge is rebuilt from the current system and
  // the solve is repeated from the caller's initial guess in this call.
  if ((s == SDSL_ERR_NOT_CONVERGED || s == SDSL_ERR_BREAKDOWN) && reused && h->opt.refactor_ratio > 0.0) {
    discarded = h->stats.iters;
    const double ms_first = h->stats.ms_solve;
    TRY(factor_impl(h));
    rebuilt = 1;
    s = solve_attempt(h, x0_zero, st);
    h->stats.ms_solve += ms_first;
  }
  // Filter relaxation (Sec. 4.3): a solve that fails under a freshly built
  // preconditioner is repeated once with a preconditioner rebuilt at the
  // relaxed threshold tau * tau_relax; later builds return to the scheduled tau.
  if ((s == SDSL_ERR_NOT_CONVERGED || s == SDSL_ERR_BREAKDOWN) && (!reused || rebuilt) &&
      h->opt.tau_relax > 0.0 && h->tau_built > 0.0) {
    discarded += h->stats.iters;
    const double ms_before = h->stats.ms_solve;
    const double scheduled = h->tau_next;
    h->tau_next = h->tau_built * h->opt.tau_relax;
    sdsl_status f = factor_impl(h);
    h->tau_next = scheduled;
    TRY(f);
    rebuilt = 1;
    s = solve_attempt(h, x0_zero, st);
    h->stats.ms_solve += ms_before;
  }
  h->solves_since_build += 1;
  TRY(to_host(h, x, h->x, h->N));
  TRY(sync(h, "solve copy-out"));
  h->stats.rebuilt = rebuilt;
  h->stats.iters_discarded = discarded;
  h->stats.status = s;  // also for early error returns (e.g. SDSL_ERR_TIMEOUT)
  // Reuse rule, slow branch: the first converged solve after a build sets
  // the baseline; a later converged solve that needs more than ratio times
  // as many iterations requests a rebuild before the next solve.  A solve
  // that did not converge never becomes the baseline: with a fresh
  // preconditioner it also requests a rebuild (for the next system).
  if (h->opt.refactor_ratio > 0.0) {
    if (s == SDSL_OK) {
      if (h->iters_post_build < 0) h->iters_post_build = h->stats.iters;
      else if ((double)h->stats.iters > h->opt.refactor_ratio * (double)h->iters_post_build)
        h->need_rebuild = true;
    } else if (s == SDSL_ERR_NOT_CONVERGED || s == SDSL_ERR_BREAKDOWN) {
      h->need_rebuild = true;
    }
  }
  if (st) *st = h->stats;
  return s;
}

// ========================================================================= ABI

extern "C" {

void sdsl_default_options(sdsl_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->form = SDSL_FORM_NORMAL;
  o->method = SDSL_BJ_PCG;
  o->nblocks = 1;
  o->tau = 1e-3;
  o->delta = 1e-12;
  o->rho = 1e-6;
  o->factor_prec = 64;
  o->rtol = 1e-8;
  o->maxit = 2000;
  o->restart = 30;
  o->refactor_ratio = 1.5;
  o->mem_space = SDSL_MEM_DEVICE;
  o->graph_iters = 16;
  o->tune = 1;
  o->apply_prec = 0;
  o->flexible = -1;
  o->orthog = 0;
  o->sweep_warps = 0;
  o->sweep_backoff_ns = -1;
  o->sweep_lane_entries = 0;
  o->sweep_wait = 0;
  o->schur_lu = 0;
}

const char* sdsl_status_str(sdsl_status s) {
  switch (s) {
    case SDSL_OK: return "ok";
    case SDSL_ERR_ARG: return "invalid argument";
    case SDSL_ERR_OOM: return "out of device memory";
    case SDSL_ERR_CUDA: return "CUDA error";
    case SDSL_ERR_BREAKDOWN: return "breakdown";
    case SDSL_ERR_NOT_CONVERGED: return "not converged";
    case SDSL_ERR_TIMEOUT: return "device wait timed out";
    case SDSL_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* sdsl_last_error(void) { return g_err.c_str(); }

int64_t sdsl_kernel_launches(void) { return (int64_t)launches_so_far(); }

sdsl_status sdsl_free(sdsl_handle h) {
  if (!h) return SDSL_OK;
  destroy_graph(h);
  if (h->st) {
    h->pc.release();
    h->sys.release();
    cudaStreamSynchronize(h->st);
  }
  if (h->h_state) cudaFreeHost(h->h_state);
  if (h->ev_a) cudaEventDestroy(h->ev_a);
  if (h->ev_b) cudaEventDestroy(h->ev_b);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (cudaEvent_t e : h->prof_ev)
    if (e) cudaEventDestroy(e);
  if (h->st) cudaStreamDestroy(h->st);
  delete h;
  return SDSL_OK;
}

sdsl_status sdsl_setup(const sdsl_options* opt, int64_t m, int64_t n, const int64_t* rowptr, const int32_t* col,
                       const double* val, const double* theta, sdsl_handle* out) {
  if (!out) return fail(SDSL_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!opt) return fail(SDSL_ERR_ARG, "options are NULL");
  if (m < 0 || n < 0 || m >= INT32_MAX || n >= INT32_MAX) return fail(SDSL_ERR_ARG, "m, n must be in [0, 2^31-1)");
  if (opt->form < SDSL_FORM_CSR || opt->form > SDSL_FORM_AUGMENTED) return fail(SDSL_ERR_ARG, "unknown form");
  if (opt->method != SDSL_BJ_PCG && !bbd_method(opt->method) && opt->method != SDSL_BJ_BICGSTAB)
    return fail(SDSL_ERR_ARG, "unknown method");
  if (opt->factor_prec != 64 && opt->factor_prec != 32 && opt->factor_prec != 16)
    return fail(SDSL_ERR_ARG, "factor_prec must be 64, 32 or 16");
  if (opt->factor_prec == 16 && bbd_method(opt->method))
    return fail(SDSL_ERR_ARG, "BF16 factors are for the Block-Jacobi methods");
  if (opt->factor_prec == 16 && opt->apply_prec == 64)
    return fail(SDSL_ERR_ARG, "BF16 factors are applied in float-float (48) or FP32 (32) arithmetic");
  if (opt->solve_kernel < 0 || opt->solve_kernel > 3) return fail(SDSL_ERR_ARG, "solve_kernel must be 0..3");
  if (opt->spmv_form < 0 || opt->spmv_form > 3) return fail(SDSL_ERR_ARG, "spmv_form must be in 0..3");
  if (opt->orthog < 0 || opt->orthog > 1) return fail(SDSL_ERR_ARG, "orthog must be 0 or 1");
  if (opt->sweep_warps < 0 || opt->sweep_warps > 16) return fail(SDSL_ERR_ARG, "sweep_warps must be in 0..16");
  if (opt->sweep_backoff_ns < -1 || opt->sweep_backoff_ns > 1000)
    return fail(SDSL_ERR_ARG, "sweep_backoff_ns must be in -1..1000");
  if (opt->sweep_lane_entries < 0 || opt->sweep_lane_entries > 64)
    return fail(SDSL_ERR_ARG, "sweep_lane_entries must be in 0..64");
  if (opt->sweep_wait < 0 || opt->sweep_wait > 3) return fail(SDSL_ERR_ARG, "sweep_wait must be in 0..3");
  if (opt->sweep_wait == 3 && opt->wait_test)
    return fail(SDSL_ERR_ARG, "wait_test exercises the barrier waits, which the level-synchronous sweep has none of");
  if (opt->schur_lu < 0 || opt->schur_lu > 2) return fail(SDSL_ERR_ARG, "schur_lu must be in 0..2");
  if (opt->wait_limit < 0) return fail(SDSL_ERR_ARG, "wait_limit must be >= 0");
  if (opt->tau_switch_step < 0 || !(opt->tau_after >= 0.0) || !(opt->tau_relax >= 0.0) || opt->tau_relax >= 1.0)
    return fail(SDSL_ERR_ARG, "tau_switch_step >= 0, tau_after >= 0 and 0 <= tau_relax < 1 are required");
  if (opt->wait_test < 0 || opt->wait_test > 1) return fail(SDSL_ERR_ARG, "wait_test must be 0 or 1");
  if (opt->sweep_slots != 0 && (opt->sweep_slots < 2 || opt->sweep_slots > 4))
    return fail(SDSL_ERR_ARG, "sweep_slots must be 0 (auto) or in 2..4");
  if (opt->sweep_far_gap < 0 || opt->sweep_far_gap > 16 || (opt->sweep_far_gap == 1 && opt->sweep_wait != 1))
    return fail(SDSL_ERR_ARG, "sweep_far_gap must be 0 (auto) or in 2..16 (1 with per-value readiness)");
  if (opt->apply_prec != 0 && opt->apply_prec != 64 && opt->apply_prec != 48 && opt->apply_prec != 32)
    return fail(SDSL_ERR_ARG, "apply_prec must be 0, 32, 48 or 64");
  if (opt->factor_prec == 64 && (opt->apply_prec == 32 || opt->apply_prec == 48))
    return fail(SDSL_ERR_ARG, "an FP32 or float-float apply needs FP32 factors (factor_prec 32)");
  if (!(opt->tau >= 0.0) || !(opt->delta >= 0.0) || !(opt->rtol > 0.0) || opt->maxit < 0)
    return fail(SDSL_ERR_ARG, "tau, delta must be >= 0, rtol > 0, maxit >= 0");
  if (opt->form == SDSL_FORM_CSR && m != n) return fail(SDSL_ERR_ARG, "CSR form needs a square matrix");
  if (opt->form != SDSL_FORM_CSR && !theta) return fail(SDSL_ERR_ARG, "theta is NULL");
  if (opt->form == SDSL_FORM_AUGMENTED && !bbd_method(opt->method))
    return fail(SDSL_ERR_ARG, "the augmented (indefinite) form needs the BBD-GMRES method");
  if (bbd_method(opt->method) && opt->form != SDSL_FORM_AUGMENTED)
    return fail(SDSL_ERR_ARG, "BBD-GMRES is implemented for the augmented form");
  const int64_t nb = opt->nblocks < 1 ? 1 : opt->nblocks;
  const int64_t dimS = opt->form == SDSL_FORM_AUGMENTED ? m + n : m;
  if (opt->form == SDSL_FORM_AUGMENTED) {
    if (opt->border < 0 || opt->border > m) return fail(SDSL_ERR_ARG, "border must be in [0, m]");
    TRY(check_block_ptr(opt->block_ptr, nb, m - opt->border));
    TRY(check_block_ptr(opt->col_block_ptr, nb, n));
  } else if (opt->block_ptr) {
    TRY(check_block_ptr(opt->block_ptr, nb, dimS));
  }
  int dev = 0;
  cudaGetDevice(&dev);
  ensure_pool(dev);
  sdsl_handle h = new sdsl_handle_s();
  h->opt = *opt;
  h->opt.nblocks = nb;
  h->dev = dev;
  cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  h->user = (cudaStream_t)opt->stream;
  if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&h->ev_a) != cudaSuccess || cudaEventCreate(&h->ev_b) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&h->prof_ev[0]) != cudaSuccess || cudaEventCreate(&h->prof_ev[1]) != cudaSuccess ||
      cudaEventCreate(&h->prof_ev[2]) != cudaSuccess || cudaEventCreate(&h->prof_ev[3]) != cudaSuccess) {
    sdsl_free(h);
    return fail(SDSL_ERR_CUDA, "stream/event creation failed");
  }
  h->sys.st = h->pc.st = h->st;
  h->sys.track(&h->live_bytes, &h->peak_bytes);
  h->pc.track(&h->live_bytes, &h->peak_bytes);
  h->form = opt->form;
  h->method = opt->method;
  h->m = m;
  h->n = n;
  h->N = dimS;
  h->nblocks = nb;
  h->border = opt->form == SDSL_FORM_AUGMENTED ? opt->border : 0;
  h->tau_next = opt->tau;
  sdsl_status s = SDSL_OK;
  {
    Scope scope(h);
    cudaEventRecord(h->ev_a, h->st);
    auto body = [&]() -> sdsl_status {
      TRY(h->sys.get(&h->flag, 4));
      TRY(h->sys.get(&h->scan_scratch, scan_scratch_elems(std::max<int64_t>(h->N, n) + 1) + 8));
      if (h->form == SDSL_FORM_CSR) {
        TRY(load_csr(h, m, m, rowptr, col, val, &h->s_rp, &h->s_ci, &h->s_v, &h->s_nnz));
      } else {
        TRY(load_csr(h, m, n, rowptr, col, val, &h->a_rp, &h->a_ci, &h->a_v, &h->a_nnz));
        TRY(h->sys.get(&h->theta, n));
        TRY(to_dev(h, h->theta, theta, n));
        TRY(transpose_input(h));
        if (h->form == SDSL_FORM_NORMAL) TRY(form_normal(h));
        else TRY(form_augmented(h, opt->block_ptr, opt->col_block_ptr));
      }
      if (h->form != SDSL_FORM_AUGMENTED) {
        h->h_bp.resize(nb + 1);
        if (opt->block_ptr) {
          std::memcpy(h->h_bp.data(), opt->block_ptr, sizeof(int64_t) * (nb + 1));
        } else {
          for (int64_t k = 0; k <= nb; ++k) h->h_bp[k] = (k * dimS) / nb;
        }
        TRY(h->sys.get(&h->d_bp, nb + 1));
        TRY(to_dev(h, h->d_bp, h->h_bp.data(), nb + 1));
      }
      TRY(h->sys.get(&h->row_block, h->N));
      TRY(h->sys.get(&h->dvals, h->N));
      TRY_CUDA(row_blocks(h->N, nb, h->d_bp, h->row_block, h->st));
      TRY(alloc_workspace(h));
      cudaEventRecord(h->ev_b, h->st);
      return sync(h, "setup end");
    };
    s = body();
  }
  if (s != SDSL_OK) {
    std::string msg = g_err;
    sdsl_free(h);
    g_err = msg;
    return s;
  }
  h->stats.ms_setup = elapsed(h);
  h->stats.n = h->N;
  h->stats.nnz_system = h->s_nnz;
  *out = h;
  return SDSL_OK;
}

sdsl_status sdsl_factor(sdsl_handle h) {
  if (!h) return fail(SDSL_ERR_ARG, "handle is NULL");
  Scope scope(h);
  return factor_impl(h);
}

sdsl_status sdsl_set_tau(sdsl_handle h, double tau) {
  if (!h) return fail(SDSL_ERR_ARG, "handle is NULL");
  if (!(tau >= 0.0)) return fail(SDSL_ERR_ARG, "tau must be >= 0");
  h->tau_next = tau;
  return SDSL_OK;
}

sdsl_status sdsl_update_diag(sdsl_handle h, const double* theta) {
  if (!h) return fail(SDSL_ERR_ARG, "handle is NULL");
  if (h->form == SDSL_FORM_CSR) return fail(SDSL_ERR_STATE, "update_diag needs the normal or augmented form");
  if (!theta) return fail(SDSL_ERR_ARG, "theta is NULL");
  Scope scope(h);
  // two-phase filter (Sec. 4.3): from IPM step tau_switch_step on, builds use tau_after
  h->ipm_step += 1;
  if (h->opt.tau_switch_step > 0 && h->ipm_step == h->opt.tau_switch_step) h->tau_next = h->opt.tau_after;
  cudaEventRecord(h->ev_a, h->st);
  TRY(to_dev(h, h->theta, theta, h->n));
  if (h->form == SDSL_FORM_NORMAL)
    TRY_CUDA(normal_values(h->m, h->a_rp, h->a_ci, h->a_v, h->at_rp, h->at_ci, h->at_v, h->theta, h->opt.rho, h->s_rp,
                           h->s_ci, h->s_v, h->st));
  else
    TRY_CUDA(augmented_theta(h->n, h->theta, h->xdiag, h->s_v, h->st));
  cudaEventRecord(h->ev_b, h->st);
  TRY(sync(h, "update_diag"));
  h->stats.ms_update = elapsed(h);
  return SDSL_OK;
}

sdsl_status sdsl_solve(sdsl_handle h, const double* b, double* x, int x0_zero, sdsl_stats* st) {
  if (!h) return fail(SDSL_ERR_ARG, "handle is NULL");
  if (!b || !x) return fail(SDSL_ERR_ARG, "b or x is NULL");
  if (!h->factored) return fail(SDSL_ERR_STATE, "sdsl_solve before sdsl_factor");
  Scope scope(h);
  int rebuilt = 0;
  TRY(solve_prepare(h, b, x, x0_zero, &rebuilt));
  const bool reused = h->solves_since_build > 0;
  sdsl_status s = solve_attempt(h, x0_zero, st);
  return solve_conclude(h, x, x0_zero, st, s, reused, rebuilt);
}

sdsl_status sdsl_batch_create(int graph_iters, sdsl_batch* out) {
  if (!out) return fail(SDSL_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (graph_iters < 0) return fail(SDSL_ERR_ARG, "graph_iters must be >= 0");
  sdsl_batch B = new sdsl_batch_s();
  cudaGetDevice(&B->dev);
  cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, B->dev);
  B->graph_iters = graph_iters;
  if (cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete B;
    return fail(SDSL_ERR_CUDA, "stream creation failed");
  }
  B->ar.st = B->st;
  *out = B;
  return SDSL_OK;
}

int sdsl_batch_size(sdsl_batch B) { return B ? (int)B->members.size() : 0; }

sdsl_status sdsl_batch_add(sdsl_batch B, sdsl_handle h, const double* b, double* x, int x0_zero) {
  if (!B || !h || !b || !x) return fail(SDSL_ERR_ARG, "NULL argument");
  if (!h->factored) return fail(SDSL_ERR_STATE, "sdsl_batch_add before sdsl_factor");
  for (auto& mb : B->members)
    if (mb.h == h) return fail(SDSL_ERR_ARG, "the handle is already in the batch");
  sdsl_handle h0 = B->members.empty() ? h : B->members.front().h;
  if (!batchable(h, h0) || h->dev != B->dev)
    return fail(SDSL_ERR_ARG, "the handle does not fit the batch's kernel shape");
  cudaEventRecord(h->ev_join, h->user);  // after the caller's earlier work on its stream
  cudaStreamWaitEvent(h->st, h->ev_join, 0);
  sdsl_batch_s::Member mb{};
  mb.h = h;
  mb.b = b;
  mb.x = x;
  mb.x0_zero = x0_zero;
  TRY(solve_prepare(h, b, x, x0_zero, &mb.rebuilt));
  mb.reused = h->solves_since_build > 0;
  if (!batchable(h, h0)) return fail(SDSL_ERR_STATE, "a rebuild changed the handle's kernel shape");
  TRY_CUDA(cudaEventRecord(h->ev_join, h->st));
  TRY_CUDA(cudaStreamWaitEvent(B->st, h->ev_join, 0));
  TRY_CUDA(cudaEventCreate(&mb.t0));
  cudaEventRecord(mb.t0, B->st);
  sdsl_status s = batch_begin(B, mb);
  if (s != SDSL_OK) {
    cudaEventDestroy(mb.t0);
    return s;
  }
  B->members.push_back(mb);
  B->dirty = true;
  return SDSL_OK;
}

sdsl_status sdsl_batch_step(sdsl_batch B, int max_graphs, sdsl_handle* done_h, sdsl_stats* done_st, int cap,
                            int* ndone) {
  if (!B || !ndone || (cap > 0 && !done_h)) return fail(SDSL_ERR_ARG, "NULL argument");
  *ndone = 0;
  if (B->members.empty()) return SDSL_OK;
  const cudaStream_t bs = B->st;
  auto running = [&]() {
    for (auto& mb : B->members)
      if (mb.tr.state == 0) return true;
    return false;
  };
  auto any_finished = [&]() {
    for (auto& mb : B->members)
      if (mb.tr.state != 0) return true;
    return false;
  };
  for (int g = 0; g < std::max(1, max_graphs) && running() && !any_finished(); ++g) {
    if (B->dirty) TRY(batch_plan(B));
    if (B->graph) {
      TRY_CUDA(cudaGraphLaunch(B->graph, bs));
      count_launch(B->graph_kernels);
    } else {
      for (int k = 0; k < 8; ++k) TRY_CUDA(batch_iteration(B));
    }
    for (auto& mb : B->members)
      if (mb.tr.state == 0)
        TRY_CUDA(cudaMemcpyAsync(mb.h->h_state, mb.h->state, sizeof(PcgState), cudaMemcpyDeviceToHost, bs));
    TRY_CUDA(cudaStreamSynchronize(bs));
    for (auto& mb : B->members) {
      if (mb.tr.state != 0) continue;
      sdsl_handle h = mb.h;
      const PcgState hs_ = *h->h_state;
      BatchTrack& tr = mb.tr;
      if (hs_.err) { tr.state = 1; tr.result = SDSL_ERR_TIMEOUT; continue; }
      if (!hs_.done) continue;
      if (hs_.done == 3) { tr.state = 1; tr.result = SDSL_ERR_BREAKDOWN; continue; }
      if (hs_.done == 2) { tr.state = 1; tr.result = SDSL_ERR_NOT_CONVERGED; continue; }
      // recurrence converged: confirm with the true residual, or restart
      TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 0, bs));
      TRY_CUDA(cudaMemcpyAsync(h->h_state, h->state, sizeof(PcgState), cudaMemcpyDeviceToHost, bs));
      TRY_CUDA(cudaStreamSynchronize(bs));
      if (h->h_state->tr <= tr.tol2) { tr.state = 1; tr.result = SDSL_OK; continue; }
      if (h->h_state->iters >= h->opt.maxit) { tr.state = 1; tr.result = SDSL_ERR_NOT_CONVERGED; continue; }
      h->stats.restarts += 1;
      TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 1, bs));
      TRY_CUDA(precond_apply(h->M, h->r, h->z, h->p, h->part_blk, h->state, 1, bs));
      TRY_CUDA(cudaMemsetAsync(&h->state->done, 0, sizeof(int), bs));
    }
  }
  // report finished members (up to cap): statistics, the reuse rule's and
  // relaxation's repeats on the member's own stream, x copied out
  std::vector<sdsl_batch_s::Member> keep;
  for (auto& mb : B->members) {
    if (mb.tr.state == 0 || *ndone >= cap) {
      keep.push_back(mb);
      continue;
    }
    sdsl_handle h = mb.h;
    TRY_CUDA(true_residual(h->A, h->b, h->x, h->r, h->part, h->state, 0, bs));  // final FP64 true residual
    TRY_CUDA(cudaMemcpyAsync(h->h_state, h->state, sizeof(PcgState), cudaMemcpyDeviceToHost, bs));
    cudaEvent_t t1;
    TRY_CUDA(cudaEventCreate(&t1));
    cudaEventRecord(t1, bs);
    TRY_CUDA(cudaStreamSynchronize(bs));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, mb.t0, t1);
    cudaEventDestroy(t1);
    cudaEventDestroy(mb.t0);
    sdsl_stats& S = h->stats;
    S.iters = h->h_state->iters;
    S.rel_res_true = mb.tr.bnorm2 > 0.0 ? std::sqrt(h->h_state->tr / mb.tr.bnorm2) : 0.0;
    S.rel_res_rec = mb.tr.bnorm2 > 0.0 ? std::sqrt(h->h_state->rr / mb.tr.bnorm2) : 0.0;
    S.status = mb.tr.result;
    S.ms_solve = ms;
    TRY_CUDA(cudaEventRecord(h->ev_join, bs));
    TRY_CUDA(cudaStreamWaitEvent(h->st, h->ev_join, 0));
    sdsl_stats out{};
    solve_conclude(h, mb.x, mb.x0_zero, &out, mb.tr.result, mb.reused, mb.rebuilt);
    cudaEventRecord(h->ev_join, h->st);  // the caller's stream sees the result
    cudaStreamWaitEvent(h->user, h->ev_join, 0);
    done_h[*ndone] = h;
    if (done_st) done_st[*ndone] = out;
    *ndone += 1;
    B->dirty = true;
  }
  B->members.swap(keep);
  return SDSL_OK;
}

sdsl_status sdsl_batch_free(sdsl_batch B) {
  if (!B) return SDSL_OK;
  for (auto& mb : B->members) cudaEventDestroy(mb.t0);
  if (B->graph) cudaGraphExecDestroy(B->graph);
  B->ar.release();
  cudaStreamSynchronize(B->st);
  cudaStreamDestroy(B->st);
  delete B;
  return SDSL_OK;
}

sdsl_status sdsl_batch_solve(int count, sdsl_handle* hs, const double* const* b, double* const* x, int x0_zero,
                             sdsl_stats* st) {
  if (count < 0) return fail(SDSL_ERR_ARG, "count must be >= 0");
  if (count == 0) return SDSL_OK;
  if (!hs || !b || !x) return fail(SDSL_ERR_ARG, "hs, b or x is NULL");
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !b[i] || !x[i]) return fail(SDSL_ERR_ARG, "a handle, b or x is NULL");
    if (!hs[i]->factored) return fail(SDSL_ERR_STATE, "sdsl_batch_solve before sdsl_factor");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(SDSL_ERR_ARG, "a handle appears twice in the batch");
  }
  bool together = count > 1;
  for (int i = 0; i < count; ++i) together = together && batchable(hs[i], hs[0]);
  sdsl_status first = SDSL_OK;
  if (!together) {  // one at a time, each in its own call
    for (int i = 0; i < count; ++i) {
      const sdsl_status s = sdsl_solve(hs[i], b[i], x[i], x0_zero, st ? &st[i] : nullptr);
      if (s != SDSL_OK && first == SDSL_OK) first = s;
    }
    return first;
  }
  sdsl_batch B = nullptr;
  TRY(sdsl_batch_create(hs[0]->opt.graph_iters, &B));
  struct Free {
    sdsl_batch b;
    ~Free() { sdsl_batch_free(b); }
  } free_b{B};
  for (int i = 0; i < count; ++i) TRY(sdsl_batch_add(B, hs[i], b[i], x[i], x0_zero));
  std::vector<sdsl_handle> dh(count);
  std::vector<sdsl_stats> ds(count);
  while (sdsl_batch_size(B) > 0) {
    int nd = 0;
    TRY(sdsl_batch_step(B, 1 << 30, dh.data(), ds.data(), count, &nd));
    for (int k = 0; k < nd; ++k) {
      for (int i = 0; i < count; ++i)
        if (hs[i] == dh[k]) {
          if (st) st[i] = ds[k];
          if (ds[k].status != SDSL_OK && first == SDSL_OK) first = (sdsl_status)ds[k].status;
        }
    }
  }
  if (first != SDSL_OK) return fail(first, "a solve of the batch did not succeed");
  return SDSL_OK;
}

sdsl_status sdsl_get_stats(sdsl_handle h, sdsl_stats* st) {
  if (!h || !st) return fail(SDSL_ERR_ARG, "NULL argument");
  *st = h->stats;
  return SDSL_OK;
}

sdsl_status sdsl_get_info(sdsl_handle h, sdsl_info* info) {
  if (!h || !info) return fail(SDSL_ERR_ARG, "NULL argument");
  info->n = h->N;
  info->nnz_system = h->s_nnz;
  info->nnz_precond = h->factored ? h->p_nnz : 0;
  info->nblocks = h->nblocks;
  info->border = h->border;
  info->levels_lower = h->factored ? h->tot_lo : 0;
  info->levels_upper = h->factored ? h->tot_up : 0;
  info->factored = h->factored ? 1 : 0;
  info->device_bytes = h->live_bytes;
  info->peak_device_bytes = h->peak_bytes;
  return SDSL_OK;
}

sdsl_status sdsl_export_system(sdsl_handle h, int64_t* rowptr, int32_t* col, double* val) {
  if (!h) return fail(SDSL_ERR_ARG, "handle is NULL");
  Scope scope(h);
  if (rowptr) TRY(to_host(h, rowptr, h->s_rp, h->N + 1));
  if (col) TRY(to_host(h, col, h->s_ci, h->s_nnz));
  if (val) TRY(to_host(h, val, h->s_v, h->s_nnz));
  return sync(h, "export system");
}

sdsl_status sdsl_export_precond(sdsl_handle h, int64_t* rowptr, int32_t* col, double* pval, double* fval,
                                double* alpha) {
  if (!h) return fail(SDSL_ERR_ARG, "handle is NULL");
  if (!h->factored) return fail(SDSL_ERR_STATE, "no preconditioner yet");
  Scope scope(h);
  if (rowptr) TRY(to_host(h, rowptr, h->p_rp, h->N + 1));
  if (col) TRY(to_host(h, col, h->p_ci, h->p_nnz));
  if (pval) TRY(to_host(h, pval, h->p_v, h->p_nnz));
  if (fval) {
    if (h->Ff) {
      std::vector<float> tmp(h->p_nnz);
      TRY(to_host(h, tmp.data(), h->Ff, h->p_nnz));
      TRY(sync(h, "export factor"));
      for (int64_t i = 0; i < h->p_nnz; ++i) fval[i] = tmp[i];
    } else {
      TRY(to_host(h, fval, h->F, h->p_nnz));
    }
  }
  if (alpha) std::memcpy(alpha, h->h_alpha.data(), sizeof(double) * h->nblocks);
  return sync(h, "export precond");
}

sdsl_status sdsl_export_levels(sdsl_handle h, int which, int32_t* nlev, int64_t* level_ptr, int32_t* level_rows) {
  if (!h) return fail(SDSL_ERR_ARG, "handle is NULL");
  if (!h->factored) return fail(SDSL_ERR_STATE, "no preconditioner yet");
  if (which != 0 && which != 1) return fail(SDSL_ERR_ARG, "which must be 0 or 1");
  Scope scope(h);
  const std::vector<int32_t>& nl = which == 0 ? h->h_nlev_lo : h->h_nlev_up;
  const int64_t tot = which == 0 ? h->tot_lo : h->tot_up;
  if (nlev) std::memcpy(nlev, nl.data(), sizeof(int32_t) * h->nblocks);
  if (level_ptr) {
    std::vector<int32_t> tmp(tot + 1);
    TRY(to_host(h, tmp.data(), which == 0 ? h->lev_ptr_lo : h->lev_ptr_up, tot + 1));
    TRY(sync(h, "export levels"));
    for (int64_t i = 0; i <= tot; ++i) level_ptr[i] = tmp[i];
  }
  if (level_rows) TRY(to_host(h, level_rows, which == 0 ? h->lev_rows_lo : h->lev_rows_up, h->h_bp[h->nblocks]));
  return sync(h, "export levels");
}

sdsl_status sdsl_export_schur(sdsl_handle h, double* sb) {
  if (!h || !sb) return fail(SDSL_ERR_ARG, "NULL argument");
  if (!bbd_method(h->method) || !h->factored) return fail(SDSL_ERR_STATE, "no Schur complement (BBD, factored)");
  Scope scope(h);
  if (h->nbord > 0) TRY(to_host(h, sb, h->SB, h->nbord * h->nbord));
  return sync(h, "export schur");
}

sdsl_status sdsl_export_schur_lu(sdsl_handle h, int32_t* ipiv, double* pivots) {
  if (!h) return fail(SDSL_ERR_ARG, "handle is NULL");
  if (!bbd_method(h->method) || !h->factored) return fail(SDSL_ERR_STATE, "no Schur complement (BBD, factored)");
  Scope scope(h);
  const int64_t m = h->nbord;
  if (m == 0) return SDSL_OK;
  if (ipiv) TRY(to_host(h, ipiv, h->ipiv, m));
  if (pivots) {
    if (h->opt.schur_lu != 2) {
      TRY(to_host(h, pivots, h->udiag, m));
    } else {  // the unblocked FP32 LU: its diagonal, widened
      std::vector<float> d(m);
      for (int64_t k = 0; k < m; ++k) TRY(to_host(h, &d[k], h->LU32 + k * m + k, 1));
      TRY(sync(h, "export schur lu"));
      for (int64_t k = 0; k < m; ++k) pivots[k] = d[k];
    }
  }
  return sync(h, "export schur lu");
}

sdsl_status sdsl_spmv(sdsl_handle h, const double* x, double* y) {
  if (!h || !x || !y) return fail(SDSL_ERR_ARG, "NULL argument");
  Scope scope(h);
  SpmvPlan A = h->A;
  if (!h->factored) {
    A.n = h->N; A.rp = h->s_rp; A.ci = h->s_ci; A.v = h->s_v; A.lanes = 32; A.grid = h->sms * 4;
  }
  TRY_CUDA(spmv(A, x, y, h->st));
  return SDSL_OK;
}

sdsl_status sdsl_precond_apply(sdsl_handle h, const double* r, double* z) {
  if (!h || !r || !z) return fail(SDSL_ERR_ARG, "NULL argument");
  if (!h->factored) return fail(SDSL_ERR_STATE, "no preconditioner yet");
  Scope scope(h);
  if (bbd_method(h->method)) return bbd_apply(h, r, z);
  TRY_CUDA(precond_apply(h->M, r, z, nullptr, h->part_blk, h->state, 2, h->st));
  return SDSL_OK;
}

}  // extern "C"
