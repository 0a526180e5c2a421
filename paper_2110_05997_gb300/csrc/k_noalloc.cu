// cpd_dgn_solve_noalloc: the uncompressed damped Gauss-Newton solve with its
// scratch memory in a fixed device array owned by this library, for callers
// that cannot hand the library a workspace.
//
// Who needs it: code that may not allocate device memory at the moment it
// wants a CPD -- for example a plugin inside a framework whose allocator owns
// all device memory, a latency-critical loop where a cudaMalloc (which can
// synchronise the device) is not acceptable, or a caller without any CUDA
// allocator of its own.  Such callers still pass their tensor and output
// buffers; everything else the solve needs lives in g_noalloc_scratch below.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds its 128 KiB until the process exits.  Host code cannot use
// the name g_noalloc_scratch as a device address (on the host it is only a
// stand-in symbol), so the first call on each device looks the address up
// with cudaGetSymbolAddress while that device is current and caches it.
#include <mutex>
#include <string.h>

#include "kernels.h"
#include "solver.cuh"

namespace cpdk {

// Capacity: result record + error history of up to kNoallocMaxIter + 1
// iterations + the balanced factors (R * sum(I_l) <= kNoallocMaxParams floats)
// + the table of CG iteration caps (kNoallocMaxIter + 1 ints).
constexpr size_t kNoallocBytes = 128 * 1024;
constexpr int kNoallocMaxIter = 4096;
constexpr int kNoallocMaxParams = 16384;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up once per device).
static cudaError_t noalloc_base(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (p == nullptr) return cudaErrorInvalidSymbol;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace cpdk

using namespace cpdk;

extern "C" int cpd_dgn_solve_noalloc(const void* T, int dtype, int L, const int64_t* dims, int R,
                                     const cpd_options* opts, const float* W0, float* W_out,
                                     float* lambda_out, cpd_info* info, void* stream) {
  // ---- validation (nothing is launched on failure) ----------------------------
  if (dims == nullptr || T == nullptr || W_out == nullptr || lambda_out == nullptr) return CPD_ERR_INVALID_ARG;
  if (L != 3 && L != 4) return CPD_ERR_UNSUPPORTED;
  if (R < 1) return CPD_ERR_INVALID_ARG;
  if (R > CPD_MAX_RANK) return CPD_ERR_UNSUPPORTED;
  if (dtype != CPD_F32 && dtype != CPD_F64) return CPD_ERR_INVALID_ARG;
  cpd_options o; cpd_default_options(&o);
  if (opts) o = *opts;
  if (o.compress != 0 || o.refine_maxiter != 0) return CPD_ERR_UNSUPPORTED;
  if (o.maxiter < 1 || !(o.tol >= 0.0) || !(o.tau >= 0.0) || !(o.cg_a >= 0.0) || !(o.cg_b >= 0.0))
    return CPD_ERR_INVALID_ARG;
  if (o.init != CPD_INIT_GIVEN && o.init != CPD_INIT_RANDOM && o.init != CPD_INIT_MLSVD)
    return CPD_ERR_INVALID_ARG;
  if (o.init == CPD_INIT_GIVEN && W0 == nullptr) return CPD_ERR_INVALID_ARG;
  if (o.block_threads < 0 || o.block_threads > 1024 || (o.block_threads % 32) != 0)
    return CPD_ERR_INVALID_ARG;
  if (!(o.mu_min >= 0.0) || o.timeout_cycles < 0) return CPD_ERR_INVALID_ARG;
  if (o.precond != CPD_PRECOND_JACOBI && o.precond != CPD_PRECOND_BLOCK) return CPD_ERR_INVALID_ARG;
  if (o.precond == CPD_PRECOND_BLOCK && R > 32) return CPD_ERR_UNSUPPORTED;
  int d[CPD_MAX_ORDER] = {1, 1, 1, 1};
  long long n = 0;
  double N = 1.0;
  for (int l = 0; l < L; ++l) {
    if (dims[l] < 1) return CPD_ERR_INVALID_ARG;
    if (dims[l] > (1 << 20)) return CPD_ERR_UNSUPPORTED;
    d[l] = (int)dims[l];
    n += (long long)R * dims[l];
    N *= (double)dims[l];
  }
  if ((double)R > N) return CPD_ERR_INVALID_ARG;
  // fixed capacity of the scratch array: larger problems are refused, not truncated
  if (o.maxiter > kNoallocMaxIter || n > kNoallocMaxParams) return CPD_ERR_WORKSPACE;
  int dev = 0, lim = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&lim, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return CPD_ERR_CUDA;
  const size_t smem = dgn_smem_bytes_host(L, d, R, 1, o.precond);
  if (N > 2.0e9 || smem > (size_t)lim) return CPD_ERR_WORKSPACE;   // T must fit the CTA's shared memory

  void* base = nullptr;
  if (noalloc_base(&base) != cudaSuccess) return CPD_ERR_CUDA;
  unsigned char* b = static_cast<unsigned char*>(base);
  DevResult* res = reinterpret_cast<DevResult*>(b);
  double* hist = reinterpret_cast<double*>(b + 256);
  float* Wc = reinterpret_cast<float*>(b + 256 + (((size_t)kNoallocMaxIter + 1) * sizeof(double) + 255) / 256 * 256);
  int* cgtab = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(Wc) + (size_t)kNoallocMaxParams * sizeof(float));
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // the result record is read back below: clear it so a failed launch cannot
  // return the previous call's outcome
  if (cudaMemsetAsync(res, 0, sizeof(DevResult), st) != cudaSuccess) return CPD_ERR_CUDA;
  DgnArgs a{};
  a.R = R;
  for (int l = 0; l < CPD_MAX_ORDER; ++l) a.dims[l] = d[l];
  a.dev_dims = nullptr;
  a.S = T; a.s_f64 = (dtype == CPD_F64);
  a.W0 = W0; a.init = o.init; a.seed = o.seed;
  a.tol = o.tol; a.tau = o.tau; a.cg_a = o.cg_a; a.cg_b = o.cg_b; a.maxiter = o.maxiter;
  a.mu0 = -1.0; a.mu_min = o.mu_min; a.precond = o.precond; a.k0 = 0;
  a.big_in_smem = 1; a.gscratch = nullptr;
  a.hist = hist; a.trace = nullptr; a.trace_cap = 0; a.trace_slot0 = 0;
  a.W_out = Wc; a.res = res;
  a.cgtab = cgtab; a.cgtab_len = o.maxiter;
  const int threads = threads_for(&o, (int)n);   // the CTA size cpd_dgn_solve launches
  if (launch_dgn_core(L, a, threads, smem, st) != cudaSuccess) return CPD_ERR_CUDA;
  long long ld[CPD_MAX_ORDER] = {1, 1, 1, 1};
  for (int l = 0; l < L; ++l) ld[l] = dims[l];
  if (launch_normalize(L, ld, R, Wc, W_out, lambda_out, st) != cudaSuccess) return CPD_ERR_CUDA;
  if (info) {
    DevResult hr;
    if (cudaMemcpyAsync(&hr, res, sizeof(DevResult), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return CPD_ERR_CUDA;
    memset(info, 0, sizeof(*info));
    info->status = hr.status; info->iters = hr.iters; info->stop_reason = hr.stop;
    info->cg_total = hr.cg_total; info->rel_err = hr.rel_err; info->mu = hr.mu;
    info->grad_inf = hr.grad_inf;
    for (int l = 0; l < L; ++l) info->core_dims[l] = d[l];
  }
  return CPD_OK;      // every launch's own status was checked above
}
