// noalloc.cu -- the normal-equation product y = A (theta o (A^T x)) + rho x
// for callers that cannot allocate device memory.
//
// Which callers, and why: a host program that hands this library device
// buffers it obtained elsewhere, from its own pool, and keeps every further
// allocation out of the process -- an interior-point driver whose memory
// manager has reserved nearly all of HBM up front (a cudaMalloc would fail
// or fragment that reservation), or a latency-bound serving loop in which a
// cudaMalloc/cudaFree pair would synchronise the device.  The handle-based
// API allocates its arenas in sdsl_setup/sdsl_factor, so such callers cannot
// use it; this entry point allocates nothing.
//
// The one intermediate, u = theta o (A^T x) (n doubles), lives in the
// file-scope device array g_normal_u below instead of an arena.  The product
// itself runs the same two kernels as the factored PCG product of the
// handle API.
#include "kernels.cuh"
#include "sdsl.h"

#include <mutex>
#include <string>

namespace sdsl {
sdsl_status report_error(sdsl_status s, const std::string& msg);
}

using namespace sdsl;

namespace {

// Static scratch: SDSL_NOALLOC_MAX_COLS doubles (4 MiB).  Every GPU on which
// the library's module is loaded holds it until the process exits.  All calls
// on a device share it.
static __device__ __align__(256) double g_normal_u[SDSL_NOALLOC_MAX_COLS];

constexpr int kMaxDevices = 64;
constexpr int kRowsPerCta = 64;

std::mutex g_mu;
double* g_u_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (0 if the driver
// cannot tell).  The runtime re-creates a device's primary context after
// cudaDeviceReset, and the module -- with g_normal_u -- is loaded anew in it,
// so an address cached for the old context would be stale.  Context ids are
// never reused within a process.
unsigned long long current_context_id() {
  typedef int (*GetCurrent)(void**);
  typedef int (*GetId)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrent>(f1);
      get_id = reinterpret_cast<GetId>(f2);
    }
    cudaGetLastError();
    looked_up = true;
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
  return 0;
}

// Device address of g_normal_u on the current device (in host code the name
// g_normal_u only stands for the symbol; it is not a device address).  Looked
// up once per device and context, with that device current.
sdsl_status scratch_address(int dev, double** out, int* sms) {
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_u_addr[dev] || g_ctx_id[dev] != ctx) {
    double* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_normal_u);
    if (e != cudaSuccess)
      return report_error(SDSL_ERR_CUDA, std::string("cudaGetSymbolAddress(g_normal_u): ") + cudaGetErrorString(e));
    int n_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
      return report_error(SDSL_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
    g_sms[dev] = n_sm > 0 ? n_sm : 1;
    g_u_addr[dev] = ptr;
    g_ctx_id[dev] = ctx;
  }
  *out = g_u_addr[dev];
  *sms = g_sms[dev];
  return SDSL_OK;
}

// Only memory the kernels can read on this device is accepted.
sdsl_status check_device_ptr(const void* p, int dev, const char* name) {
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return report_error(SDSL_ERR_ARG, std::string(name) + " is not a device pointer");
  }
  const bool ok = (a.type == cudaMemoryTypeDevice && a.device == dev) || a.type == cudaMemoryTypeManaged;
  if (!ok) return report_error(SDSL_ERR_ARG, std::string(name) + " is not device memory of the current device");
  return SDSL_OK;
}

int lanes_per_row(int64_t nnz, int64_t rows) {
  const double avg = rows > 0 ? (double)nnz / (double)rows : 1.0;
  int lanes = 2;
  while (lanes < 32 && lanes * 24.0 <= avg) lanes <<= 1;
  return lanes;
}

int grid_for_rows(int64_t rows, int sms) {
  int64_t g = (rows + kRowsPerCta - 1) / kRowsPerCta;
  if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

extern "C" sdsl_status sdsl_normal_spmv_noalloc(int64_t m, int64_t n, int64_t nnz, const int64_t* a_rowptr,
                                                const int32_t* a_col, const double* a_val,
                                                const int64_t* at_rowptr, const int32_t* at_col,
                                                const double* at_val, const double* theta, double rho,
                                                const double* x, double* y, void* stream) {
  if (m < 0 || n < 0 || nnz < 0) return report_error(SDSL_ERR_ARG, "m, n and nnz must be >= 0");
  if (n > SDSL_NOALLOC_MAX_COLS)
    return report_error(SDSL_ERR_ARG, "n = " + std::to_string(n) + " exceeds the no-alloc scratch limit of " +
                                          std::to_string((long long)SDSL_NOALLOC_MAX_COLS) + " columns");
  if (m > INT32_MAX || nnz > INT32_MAX)
    return report_error(SDSL_ERR_ARG, "m and nnz must fit the int32 column indices");
  if (m == 0) return SDSL_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_error(SDSL_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report_error(SDSL_ERR_ARG, "device ordinal beyond 63");
  struct Arg { const void* p; const char* name; bool needed; };
  const Arg args[] = {{a_rowptr, "a_rowptr", true}, {a_col, "a_col", nnz > 0}, {a_val, "a_val", nnz > 0},
                      {at_rowptr, "at_rowptr", n > 0}, {at_col, "at_col", nnz > 0 && n > 0},
                      {at_val, "at_val", nnz > 0 && n > 0}, {theta, "theta", n > 0}, {x, "x", true},
                      {y, "y", true}};
  for (const Arg& a : args) {
    if (!a.needed) continue;
    if (!a.p) return report_error(SDSL_ERR_ARG, std::string(a.name) + " is NULL");
    sdsl_status s = check_device_ptr(a.p, dev, a.name);
    if (s != SDSL_OK) return s;
  }
  double* u = nullptr;
  int sms = 1;
  sdsl_status s = scratch_address(dev, &u, &sms);
  if (s != SDSL_OK) return s;

  SpmvPlan A{};
  A.n = m;
  A.factored = 1;
  A.ncols = n;
  A.a_rp = a_rowptr; A.a_ci = a_col; A.a_v = a_val;
  A.at_rp = at_rowptr; A.at_ci = at_col; A.at_v = at_val;
  A.theta = theta;
  A.rho = rho;
  A.u = u;  // every u[j], j < n, is written by the first kernel before the second reads it
  A.a_lanes = lanes_per_row(nnz, m);
  A.at_lanes = lanes_per_row(nnz, n);
  A.grid = grid_for_rows(m, sms);
  A.at_grid = grid_for_rows(n, sms);
  e = factored_product(A, x, y, nullptr, nullptr, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) return report_error(SDSL_ERR_CUDA, std::string("normal product launch: ") + cudaGetErrorString(e));
  return SDSL_OK;
}
