// C ABI of libcpd: validation, workspace carving and the launch sequence of
// the method (Fig. "tensorfox-flow" of the thesis).  No allocation happens
// here; every buffer is the caller's.
#include <mutex>
#include <string.h>
#include <vector>

#include "kernels.h"
#include "solver.cuh"

using namespace cpdk;

namespace {

struct Carver {
  char* base; size_t cap; size_t used = 0; bool ok = true;
  Carver(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
  template <typename T> T* take(size_t count) {
    size_t at = (used + 255) & ~(size_t)255;
    size_t bytes = count * sizeof(T);
    used = at + bytes;
    if (base == nullptr) return nullptr;            // sizing pass
    if (used > cap) { ok = false; return nullptr; }
    return reinterpret_cast<T*>(base + at);
  }
};

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

bool pass_ok(int L, const int64_t* dims, int R) {
  long long d[CPD_MAX_ORDER] = {1, 1, 1, 1};
  for (int l = 0; l < L && l < CPD_MAX_ORDER; ++l) d[l] = dims[l];
  return refine_pass_supported(L, d, R);
}

int validate_common(int L, const int64_t* dims, int R) {
  if (dims == nullptr) return CPD_ERR_INVALID_ARG;
  if (L < 1 || R < 1) return CPD_ERR_INVALID_ARG;
  if (L != 3 && L != 4) return CPD_ERR_UNSUPPORTED;
  if (R > CPD_MAX_RANK) return CPD_ERR_UNSUPPORTED;
  double N = 1.0;
  for (int l = 0; l < L; ++l) {
    if (dims[l] < 1) return CPD_ERR_INVALID_ARG;
    if (dims[l] > (1 << 20)) return CPD_ERR_UNSUPPORTED;
    N *= (double)dims[l];
  }
  if (N > 4.0e9) return CPD_ERR_UNSUPPORTED;
  if ((double)R > N) return CPD_ERR_INVALID_ARG;
  return CPD_OK;
}

// The single-CTA solver (dGN on T itself, compress = 0) indexes the tensor
// with 32-bit integers: larger tensors are refused before anything is sized.
bool uncompressed_fits(int L, const int64_t* dims) {
  double N = 1.0;
  for (int l = 0; l < L; ++l) N *= (double)dims[l];
  return N <= (double)(0x7fffffff - 1024);
}

// dGN with every iteration one pass over T (Sec. 4.9: uncompressed CPDs of
// large tensors): no compression, an FP32 tensor of at least 2^20 entries,
// a random or given start, and a shape the refinement pass covers.  The
// single-CTA and cluster solvers hold T (or its slices) in shared memory and
// stay the path for smaller tensors and for the MLSVD-energy start.
constexpr double kFullMinEntries = 1048576.0;
bool full_mode(int L, const int64_t* dims, int R, const cpd_options& o, int dtype) {
  if (o.compress || dtype != CPD_F32) return false;
  if (o.init != CPD_INIT_RANDOM && o.init != CPD_INIT_GIVEN) return false;
  double N = 1.0;
  for (int l = 0; l < L; ++l) N *= (double)dims[l];
  return N >= kFullMinEntries && pass_ok(L, dims, R);
}

int validate_options(const cpd_options* o) {
  if (o == nullptr) return CPD_OK;
  if (o->maxiter < 1 || o->maxiter > 100000) return CPD_ERR_INVALID_ARG;
  if (!(o->tol >= 0.0) || !(o->tau >= 0.0) || !(o->mlsvd_tol >= 0.0)) return CPD_ERR_INVALID_ARG;
  if (!(o->cg_a >= 0.0) || !(o->cg_b >= 0.0)) return CPD_ERR_INVALID_ARG;
  if (o->init < CPD_INIT_MLSVD || o->init > CPD_INIT_GIVEN) return CPD_ERR_INVALID_ARG;
  if (o->gram_precision != CPD_GRAM_FP32 && o->gram_precision != CPD_GRAM_BF16) return CPD_ERR_INVALID_ARG;
  if (o->refine_maxiter < 0 || o->refine_maxiter > 100000) return CPD_ERR_INVALID_ARG;
  if (o->block_threads < 0 || o->block_threads > 1024 || (o->block_threads % 32) != 0)
    return CPD_ERR_INVALID_ARG;
  if (!(o->mu_min >= 0.0) || o->timeout_cycles < 0) return CPD_ERR_INVALID_ARG;
  if (o->precond != CPD_PRECOND_JACOBI && o->precond != CPD_PRECOND_BLOCK) return CPD_ERR_INVALID_ARG;
  return CPD_OK;
}

// Largest dynamic shared memory per CTA this device grants (opt-in).
size_t smem_limit() {
  static size_t lim = 0;
  if (lim == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && v > 0)
      lim = (size_t)v;
    else
      lim = 227 * 1024;
  }
  return lim;
}

// Everything the solve needs, carved from the workspace (or sized when base == nullptr).
struct SolvePlan {
  int L, R, dtype;
  int full = 0;                 // every dGN iteration a pass over T (full_mode)
  long long dims[CPD_MAX_ORDER];
  int idims[CPD_MAX_ORDER];
  int P[CPD_MAX_ORDER];
  int n_full;
  // device buffers
  DevResult* res = nullptr;
  int* err = nullptr;           // CPD_ERR_TIMEOUT once a bounded device wait ran out
  double* hist = nullptr;
  int* cgtab = nullptr; int cgtab_len = 0;
  float* W_core = nullptr;     // balanced factors after the core dGN (core space)
  float* W_full = nullptr;     // original space (compress path / refinement)
  float* gscratch = nullptr;
  int big_in_smem = 1;
  size_t dgn_smem = 0;
  int cluster = 0;              // CTAs of the cluster solver for a large core (0: one CTA)
  size_t cluster_smem = 0;
  // compression
  int* core_dims_dev = nullptr;
  float* U = nullptr; float* sigma = nullptr; float* G = nullptr; float* Y0 = nullptr; float* Y1 = nullptr;
  float* core = nullptr; float* eig_work = nullptr; float* W0_core = nullptr;
  float* tc_scratch = nullptr; size_t tc_scratch_bytes = 0;
  // refinement
  RefineState* rstate = nullptr; int* rdone = nullptr; double* resq = nullptr; float* rG = nullptr;
  double* rhist = nullptr; float* rvecs = nullptr; int r_vec_in_smem = 1; size_t r_smem = 0;
};

void plan_solve(SolvePlan& p, Carver& c, const cpd_options& o) {
  const int L = p.L, R = p.R;
  int cmax[CPD_MAX_ORDER];
  for (int l = 0; l < CPD_MAX_ORDER; ++l) cmax[l] = 1;
  for (int l = 0; l < L; ++l) cmax[l] = o.compress ? p.P[l] : p.idims[l];
  p.res = c.take<DevResult>(1);
  p.err = c.take<int>(1);
  p.hist = c.take<double>((size_t)o.maxiter + 1);
  p.cgtab_len = o.maxiter + o.refine_maxiter;
  p.cgtab = c.take<int>((size_t)p.cgtab_len + 1);
  Shape sc; make_shape(sc, L, cmax, R);
  p.W_core = c.take<float>(sc.n);
  // the single-CTA solver's buffers: all in shared memory, else the
  // tensor-sized ones in global scratch, else (high ranks) the vectors too
  p.big_in_smem = 1;
  if (!p.full) {
    while (p.big_in_smem > -1 && dgn_smem_bytes_host(L, cmax, R, p.big_in_smem, o.precond) > smem_limit())
      --p.big_in_smem;
    p.dgn_smem = dgn_smem_bytes_host(L, cmax, R, p.big_in_smem, o.precond);
  }
  if (p.big_in_smem <= 0) p.gscratch = c.take<float>(dgn_gscratch_floats_host(L, cmax, R, p.big_in_smem));
  // a core of 8192 entries or more (or one beyond a CTA's shared memory) is
  // solved by a cluster, each CTA holding a slice of it (FP32 tensors only)
  if (!p.full && (sc.N >= 8192 || p.big_in_smem <= 0) && (o.compress || p.dtype == CPD_F32)) {
    for (int cs : {16, 8}) {
      const size_t sm = dgn_cluster_smem_bytes_host(L, cmax, R, cs, o.precond);
      if (sm <= smem_limit() && sc.N / cmax[0] >= cs) { p.cluster = cs; p.cluster_smem = sm; break; }
    }
  }
  p.n_full = 0;
  for (int l = 0; l < L; ++l) p.n_full += R * p.idims[l];
  p.W_full = c.take<float>(p.n_full);
  if (o.compress) {
    p.core_dims_dev = c.take<int>(CPD_MAX_ORDER);
    size_t nU = 0, nS = 0, maxI = 0;
    for (int l = 0; l < L; ++l) { nU += (size_t)p.idims[l] * p.P[l]; nS += p.P[l]; maxI = maxI > (size_t)p.idims[l] ? maxI : (size_t)p.idims[l]; }
    p.U = c.take<float>(nU);
    p.sigma = c.take<float>(nS);
    p.G = c.take<float>(maxI * maxI);
    // ST intermediates: after mode l the tensor is P_1..P_l x I_{l+1}..I_L
    size_t ymax = 1;
    for (int l = 0; l < L; ++l) {
      size_t sz = 1;
      for (int j = 0; j < L; ++j) sz *= (size_t)(j <= l ? p.P[j] : p.idims[j]);
      ymax = ymax > sz ? ymax : sz;
    }
    p.Y0 = c.take<float>(ymax);
    p.Y1 = c.take<float>(ymax);
    size_t ncore = 1;
    for (int l = 0; l < L; ++l) ncore *= (size_t)p.P[l];
    p.core = c.take<float>(ncore);
    size_t ew = 0;
    for (int l = 0; l < L; ++l) { size_t w = eig_work_floats(p.idims[l], p.P[l]); ew = ew > w ? ew : w; }
    p.eig_work = c.take<float>(ew);
    p.W0_core = c.take<float>(sc.n);
    if (o.gram_precision == CPD_GRAM_BF16) {
      long long Cc = 1;
      for (int l = 1; l < L; ++l) Cc *= p.dims[l];
      p.tc_scratch_bytes = gram_bf16_tc_scratch_bytes(p.dims[0], Cc);
      p.tc_scratch = c.take<float>((p.tc_scratch_bytes + 3) / 4);
    }
  }
  if (o.refine_maxiter > 0 || p.full) {
    p.rstate = reinterpret_cast<RefineState*>(c.take<char>(refine_state_bytes()));
    p.rdone = c.take<int>(1);
    p.resq = c.take<double>(2);
    p.rG = c.take<float>(p.n_full);
    const int hmax = p.full && o.maxiter > o.refine_maxiter ? o.maxiter : o.refine_maxiter;
    p.rhist = c.take<double>((size_t)hmax + 1);
    size_t sm = refine_step_smem_bytes(L, p.dims, R, 1, o.precond);
    p.r_vec_in_smem = sm <= smem_limit() ? 1 : 0;
    p.r_smem = refine_step_smem_bytes(L, p.dims, R, p.r_vec_in_smem, o.precond);
    if (!p.r_vec_in_smem) p.rvecs = c.take<float>((size_t)p.n_full * 8 + 1024);
  }
}

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return CPD_ERR_CUDA; } while (0)
// launch under a profiling scope on the stream `st` in scope
#define PL(name, x) do { ProfScope ps_(st, name); CK(x); } while (0)

int fill_dims(SolvePlan& p, int L, const int64_t* dims, int R) {
  p.L = L; p.R = R;
  for (int l = 0; l < CPD_MAX_ORDER; ++l) { p.dims[l] = 1; p.idims[l] = 1; p.P[l] = 1; }
  for (int l = 0; l < L; ++l) {
    p.dims[l] = dims[l]; p.idims[l] = (int)dims[l];
    p.P[l] = (int)(dims[l] < R ? dims[l] : R);
  }
  return CPD_OK;
}

// Compression into p.core / p.U / p.sigma / p.core_dims_dev (Algorithm "Compression").
int run_compress(SolvePlan& p, const float* T, const cpd_options& o, cudaStream_t st) {
  const int L = p.L;
  if (o.st_mlsvd) {
    // Algorithm ST-MLSVD: Gram of the partially projected tensor, eigenpairs,
    // project, next mode.
    const float* cur = T;
    float* bufs[2] = {p.Y0, p.Y1};
    long long a_max = 1;
    size_t offU = 0, offS = 0;
    for (int l = 0; l < L; ++l) {
      long long c = 1;
      for (int j = l + 1; j < L; ++j) c *= p.dims[j];
      View3 v{1, p.dims[l], c, l > 0 ? p.core_dims_dev : nullptr, l};
      CK(cudaMemsetAsync(p.G, 0, sizeof(float) * (size_t)p.dims[l] * p.dims[l], st));
      if (l == 0 && o.gram_precision == CPD_GRAM_BF16) {
        PL("gram_bf16_tc", launch_gram_bf16_tc(T, p.dims[0], c, p.G, p.tc_scratch, p.tc_scratch_bytes, st, p.err,
                                               o.timeout_cycles));
      } else {
        PL("gram_fp32", launch_gram_simt(cur, v, a_max, p.G, st));
      }
      EigArgs ea{p.G, p.idims[l], p.P[l], p.U + offU, p.sigma + offS, p.core_dims_dev + l,
                 o.mlsvd_tol, L, o.seed + 7919ull * (uint64_t)l, p.eig_work,
                 o.gram_precision == CPD_GRAM_BF16 ? 1 : 0};
      PL("eig", launch_eig(ea, st));
      float* out = (l == L - 1) ? p.core : bufs[l & 1];
      PL(l == 0 ? "project_T" : "project",
         launch_project(cur, v, a_max, p.U + offU, p.core_dims_dev + l, p.P[l], out, st, p.err,
                        o.timeout_cycles));
      cur = out;
      a_max *= p.P[l];
      offU += (size_t)p.idims[l] * p.P[l];
      offS += p.P[l];
    }
  } else {
    // Algorithm MLSVD (classic): all Grams of T, then S = (U1^T, ..., UL^T)·T.
    size_t offU = 0, offS = 0;
    for (int l = 0; l < L; ++l) {
      long long a = 1, c = 1;
      for (int j = 0; j < l; ++j) a *= p.dims[j];
      for (int j = l + 1; j < L; ++j) c *= p.dims[j];
      View3 v{a, p.dims[l], c, nullptr, 0};
      CK(cudaMemsetAsync(p.G, 0, sizeof(float) * (size_t)p.dims[l] * p.dims[l], st));
      if (l == 0 && o.gram_precision == CPD_GRAM_BF16)
        PL("gram_bf16_tc", launch_gram_bf16_tc(T, p.dims[0], c, p.G, p.tc_scratch, p.tc_scratch_bytes, st, p.err,
                                               o.timeout_cycles));
      else
        PL("gram_fp32", launch_gram_simt(T, v, a, p.G, st));
      EigArgs ea{p.G, p.idims[l], p.P[l], p.U + offU, p.sigma + offS, p.core_dims_dev + l,
                 o.mlsvd_tol, L, o.seed + 7919ull * (uint64_t)l, p.eig_work,
                 o.gram_precision == CPD_GRAM_BF16 ? 1 : 0};
      PL("eig", launch_eig(ea, st));
      offU += (size_t)p.idims[l] * p.P[l];
      offS += p.P[l];
    }
    const float* cur = T;
    float* bufs[2] = {p.Y0, p.Y1};
    long long a_max = 1;
    offU = 0;
    for (int l = 0; l < L; ++l) {
      long long c = 1;
      for (int j = l + 1; j < L; ++j) c *= p.dims[j];
      View3 v{1, p.dims[l], c, l > 0 ? p.core_dims_dev : nullptr, l};
      float* out = (l == L - 1) ? p.core : bufs[l & 1];
      PL(l == 0 ? "project_T" : "project",
         launch_project(cur, v, a_max, p.U + offU, p.core_dims_dev + l, p.P[l], out, st, p.err,
                        o.timeout_cycles));
      cur = out;
      a_max *= p.P[l];
      offU += (size_t)p.idims[l] * p.P[l];
    }
  }
  return CPD_OK;
}

// dGN iterations on the full tensor T from the factors Wr (stacked, in place):
// each iteration one pass over T and one single-CTA step, at most `maxiter`
// of them, the state already primed (launch_refine_init); trace records from
// slot `slot0`.  While st is being captured (and `side` is given) the
// iterations are the body of a conditional while node.
int enqueue_refine(SolvePlan& p, const cpd_options& o, const void* T, int L, int R, float* Wr, int maxiter,
                   int slot0, int cgtab_len, double* trace, int trace_cap, cudaStream_t st, cudaStream_t side,
                   int* refine_loop) {
  RefinePassArgs pa{};
  pa.T = static_cast<const float*>(T); pa.L = L; pa.R = R; pa.W = Wr; pa.G = p.rG; pa.esq = p.resq;
  for (int l = 0; l < CPD_MAX_ORDER; ++l) pa.dims[l] = p.dims[l];
  pa.done = p.rdone;
  pa.err = p.err; pa.budget = o.timeout_cycles;
  RefineStepArgs sa{};
  sa.L = L; sa.R = R; sa.W = Wr; sa.G = p.rG; sa.esq = p.resq; sa.state = p.rstate;
  for (int l = 0; l < CPD_MAX_ORDER; ++l) sa.dims[l] = p.dims[l];
  sa.vecs = p.rvecs; sa.vec_in_smem = p.r_vec_in_smem; sa.maxiter = maxiter;
  sa.tol = o.tol; sa.cg_a = o.cg_a; sa.cg_b = o.cg_b; sa.mu_min = o.mu_min; sa.seed = o.seed; sa.hist = p.rhist;
  sa.trace = trace; sa.trace_cap = trace_cap; sa.trace_slot0 = slot0; sa.done = p.rdone;
  sa.cgtab = p.cgtab; sa.cgtab_len = cgtab_len;
  sa.err = p.err;
  sa.precond = o.precond;
  const int rthreads = 1024;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (side != nullptr && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive) {
    // iteration 0, then a while node whose body is one iteration; every
    // exit of the step kernel sets the condition, so the graph runs only
    // the iterations the stop tests allow (at most refine_maxiter)
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* ed = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
    sa.use_cond = 1; sa.cond = h;
    pa.want_tsq = 1; sa.j = 0;
    PL("refine_pass", launch_refine_pass(pa, st));
    PL("refine_step", launch_refine_step(sa, rthreads, p.r_smem, st));
    CK(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, &ed, &nd));
    cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, ed, nd, &np));
    CK(cudaStreamBeginCaptureToGraph(side, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    pa.want_tsq = 0; sa.j_from_state = 1;
    cudaError_t e = launch_refine_pass(pa, side);
    if (e == cudaSuccess) e = launch_refine_step(sa, rthreads, p.r_smem, side);
    cudaGraph_t body = nullptr;                 // owned by the conditional node
    const cudaError_t ee = cudaStreamEndCapture(side, &body);
    CK(e);
    CK(ee);
    CK(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    if (refine_loop) *refine_loop = 1;
  } else {
    // under profiling the host reads the stop flag after each step and
    // launches no further iterations, as the graph loop does (the stage
    // times then hold only the iterations that run)
    const bool watch = profile_enabled() && cudaStreamIsCapturing(st, &cs) == cudaSuccess &&
                       cs == cudaStreamCaptureStatusNone;
    for (int j = 0; j <= maxiter; ++j) {
      pa.want_tsq = (j == 0);
      PL("refine_pass", launch_refine_pass(pa, st));
      sa.j = j;
      PL("refine_step", launch_refine_step(sa, rthreads, p.r_smem, st));
      if (watch) {
        int done = 0;
        CK(cudaMemcpyAsync(&done, p.rdone, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (done) break;
      }
    }
  }
  return CPD_OK;
}

// The launch sequence of one solve (Fig. "tensorfox-flow"), enqueued on st.
// `side` (optional) is an idle stream on which, while st is being captured,
// the refinement iterations are captured as the body of a conditional while
// node (*refine_loop = 1); otherwise all refine_maxiter + 1 iterations are
// enqueued and the stopped ones exit at once.
int enqueue_solve(SolvePlan& p, const cpd_options& o, const void* T, int dtype, int L, int R,
                  const float* W0, float* W_out, float* lambda_out, double* trace, cudaStream_t st,
                  cudaStream_t side = nullptr, int* refine_loop = nullptr) {
  const int trace_cap = trace ? (o.maxiter + o.refine_maxiter) : 0;
  CK(cudaMemsetAsync(p.err, 0, sizeof(int), st));

  if (p.full) {
    // dGN on T itself, every iteration one pass (no core solve): the start
    // (random draws or the given factors, balanced) and mu0 = tau mean|T|,
    // then the iterations, then (refine_maxiter > 0) the refinement as the
    // method states it, a second run of iterations from where dGN stopped
    PL("full_start", launch_full_start(L, p.dims, R, o.init, W0, o.seed, o.tau, static_cast<const float*>(T),
                                       p.resq, p.W_full, p.res, p.cgtab, p.cgtab_len, o.cg_a, o.cg_b, st));
    PL("refine_init", launch_refine_init(p.rstate, p.res, p.rdone, st));
    const bool second = o.refine_maxiter > 0;
    int rc = enqueue_refine(p, o, T, L, R, p.W_full, o.maxiter, 0, p.cgtab_len, trace, trace_cap, st,
                            second ? nullptr : side, second ? nullptr : refine_loop);
    if (rc != CPD_OK) return rc;
    PL("refine_result", launch_refine_result(p.rstate, p.res, st));
    if (second) {
      PL("refine_init", launch_refine_init(p.rstate, p.res, p.rdone, st));
      rc = enqueue_refine(p, o, T, L, R, p.W_full, o.refine_maxiter, o.maxiter, p.cgtab_len, trace, trace_cap, st,
                          nullptr, nullptr);
      if (rc != CPD_OK) return rc;
    }
    PL("normalize", launch_normalize(L, p.dims, R, p.W_full, W_out, lambda_out, st));
    return CPD_OK;
  }

  // ---- compression and initial factors -----------------------------------------
  DgnArgs a{};
  a.R = R;
  for (int l = 0; l < CPD_MAX_ORDER; ++l) a.dims[l] = (l < L) ? p.idims[l] : 1;
  a.init = o.init;
  a.W0 = W0;
  if (o.compress) {
    int rc = run_compress(p, static_cast<const float*>(T), o, st);
    if (rc != CPD_OK) return rc;
    a.dev_dims = p.core_dims_dev;
    a.S = p.core;
    a.s_f64 = 0;
    if (o.init == CPD_INIT_GIVEN) {
      PL("project_given", launch_project_given(L, p.dims, R, p.U, p.core_dims_dev, p.P, W0, p.W0_core, st));
      a.W0 = p.W0_core;
    }
  } else {
    a.dev_dims = nullptr;
    a.S = T;
    a.s_f64 = dtype == CPD_F64;
  }
  a.seed = o.seed; a.tol = o.tol; a.tau = o.tau; a.cg_a = o.cg_a; a.cg_b = o.cg_b;
  a.maxiter = o.maxiter; a.mu0 = -1.0; a.mu_min = o.mu_min; a.precond = o.precond; a.k0 = 0;
  a.big_in_smem = p.big_in_smem; a.gscratch = p.gscratch;
  a.hist = p.hist; a.trace = trace; a.trace_cap = trace_cap; a.trace_slot0 = 0;
  a.W_out = p.W_core; a.res = p.res;
  a.cgtab = p.cgtab; a.cgtab_len = p.cgtab_len;
  int cmax[CPD_MAX_ORDER] = {1, 1, 1, 1};
  for (int l = 0; l < L; ++l) cmax[l] = o.compress ? p.P[l] : p.idims[l];
  Shape sc; make_shape(sc, L, cmax, R);
  if (p.cluster > 0) {
    cudaError_t ce;
    {
      ProfScope ps_(st, "dgn_core");
      ce = launch_dgn_cluster(L, a, threads_for(&o, sc.n), p.cluster, p.cluster_smem, st);
    }
    if (ce == cudaErrorInvalidConfiguration) {   // the device cannot place the cluster: one CTA
      (void)cudaGetLastError();
      PL("dgn_core", launch_dgn_core(L, a, threads_for(&o, sc.n), p.dgn_smem, st));
    } else {
      CK(ce);
    }
  } else {
    PL("dgn_core", launch_dgn_core(L, a, threads_for(&o, sc.n), p.dgn_smem, st));
  }

  // ---- uncompression, refinement, output ---------------------------------------------
  const float* Wfinal = p.W_core;
  if (o.compress) {
    PL("uncompress", launch_uncompress(L, p.dims, R, p.U, p.core_dims_dev, p.P, p.W_core, p.W_full, st));
    Wfinal = p.W_full;
  }
  if (o.refine_maxiter > 0) {
    float* Wr = p.W_full;
    if (!o.compress) CK(cudaMemcpyAsync(Wr, p.W_core, sizeof(float) * p.n_full, cudaMemcpyDeviceToDevice, st));
    PL("refine_init", launch_refine_init(p.rstate, p.res, p.rdone, st));
    const int rc = enqueue_refine(p, o, T, L, R, Wr, o.refine_maxiter, o.maxiter, p.cgtab_len, trace, trace_cap, st,
                                  side, refine_loop);
    if (rc != CPD_OK) return rc;
    Wfinal = Wr;
  }
  PL("normalize", launch_normalize(L, p.dims, R, Wfinal, W_out, lambda_out, st));

  return CPD_OK;
}

// ---- CUDA graphs of the launch sequence ----------------------------------------
// One solve is ~10 + 3 * refine_maxiter launches; replaying a captured graph
// removes the per-launch host cost.  Graphs are cached per argument set (all
// pointers, sizes and options), least recently used first out.
struct GraphKey {
  int dev, dtype, L, R;
  long long dims[CPD_MAX_ORDER];
  cpd_options o;
  const void* T; const float* W0; float* W_out; float* lam; double* trace; void* ws; size_t ws_bytes;
};
struct GraphEntry { GraphKey k; cudaGraphExec_t exec; unsigned long long used; long long kernels; int refine_loop; };
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;
unsigned long long g_graph_clock = 0;
constexpr size_t kMaxGraphs = 16;

bool same_key(const GraphKey& a, const GraphKey& b) { return memcmp(&a, &b, sizeof(GraphKey)) == 0; }

// An idle stream per thread and device for capturing graph-loop bodies
// (created before any capture begins).
cudaStream_t side_stream() {
  static thread_local cudaStream_t s[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (s[dev] == nullptr && cudaStreamCreateWithFlags(&s[dev], cudaStreamNonBlocking) != cudaSuccess) {
    s[dev] = nullptr;
    cudaGetLastError();
  }
  return s[dev];
}

}  // namespace

extern "C" {

void cpd_default_options(cpd_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->maxiter = 200;
  o->tol = 1e-6;
  o->tau = 1.0;
  o->cg_a = 0.4;
  o->cg_b = 0.9;
  o->mlsvd_tol = 1e-6;
  o->st_mlsvd = 1;
  o->compress = 1;
  o->init = CPD_INIT_MLSVD;
  o->gram_precision = CPD_GRAM_FP32;
  o->refine_maxiter = 0;
  o->seed = 0;
  o->block_threads = 0;
  o->mu_min = 1e-5;
  o->timeout_cycles = 0;
  o->precond = CPD_PRECOND_JACOBI;
}

const char* cpd_status_string(int s) {
  switch (s) {
    case CPD_OK: return "ok";
    case CPD_ERR_INVALID_ARG: return "invalid argument";
    case CPD_ERR_CUDA: return "CUDA error";
    case CPD_ERR_WORKSPACE: return "workspace too small";
    case CPD_ERR_NUMERIC: return "non-finite value in the iteration";
    case CPD_ERR_TIMEOUT: return "bounded wait expired";
    case CPD_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

size_t cpd_workspace_size(int L, const int64_t* dims, int R, const cpd_options* opts) {
  if (validate_common(L, dims, R) != CPD_OK) return 0;
  cpd_options o; cpd_default_options(&o);
  if (opts) o = *opts;
  const bool full = full_mode(L, dims, R, o, CPD_F32);
  if (!o.compress && !full && !uncompressed_fits(L, dims)) return 0;
  SolvePlan p; fill_dims(p, L, dims, R); p.dtype = CPD_F32; p.full = full ? 1 : 0;
  Carver c(nullptr, 0);
  plan_solve(p, c, o);
  if (full && uncompressed_fits(L, dims)) {     // an FP64 tensor of this shape takes the other path
    SolvePlan q; fill_dims(q, L, dims, R); q.dtype = CPD_F64;
    Carver c2(nullptr, 0);
    plan_solve(q, c2, o);
    if (c2.used > c.used) c.used = c2.used;
  }
  // component calls reuse the same workspace: make room for their scratch too
  int d[CPD_MAX_ORDER] = {1, 1, 1, 1};
  for (int l = 0; l < L; ++l) d[l] = (int)dims[l];
  size_t extra = (!uncompressed_fits(L, dims) || dgn_smem_bytes_host(L, d, R, 1) <= smem_limit())
                     ? 0 : dgn_gscratch_floats_host(L, d, R) * 4;
  size_t need = c.used + 256;
  return need > extra + 512 ? need : extra + 512;
}

int cpd_dgn_solve(const void* T, int dtype, int L, const int64_t* dims, int R,
                  const cpd_options* opts, const float* W0, float* W_out, float* lambda_out,
                  cpd_info* info, double* trace, void* workspace, size_t ws_bytes, void* stream) {
  int v = validate_common(L, dims, R);
  if (v != CPD_OK) return v;
  if ((v = validate_options(opts)) != CPD_OK) return v;
  if (T == nullptr || W_out == nullptr || lambda_out == nullptr || workspace == nullptr)
    return CPD_ERR_INVALID_ARG;
  if (dtype != CPD_F32 && dtype != CPD_F64) return CPD_ERR_INVALID_ARG;
  cpd_options o; cpd_default_options(&o);
  if (opts) o = *opts;
  if (o.init == CPD_INIT_GIVEN && W0 == nullptr) return CPD_ERR_INVALID_ARG;
  if (dtype == CPD_F64 && (o.compress || o.refine_maxiter > 0)) return CPD_ERR_UNSUPPORTED;
  if (o.gram_precision == CPD_GRAM_BF16 && !o.compress) return CPD_ERR_INVALID_ARG;
  if (o.gram_precision == CPD_GRAM_BF16 && !gram_bf16_tc_supported(dims[0], static_cast<const float*>(T)))
    return CPD_ERR_UNSUPPORTED;
  if (o.refine_maxiter > 0 && !pass_ok(L, dims, R)) return CPD_ERR_UNSUPPORTED;
  if (o.precond == CPD_PRECOND_BLOCK && R > 32) return CPD_ERR_UNSUPPORTED;
  const bool full = full_mode(L, dims, R, o, dtype);
  if (!o.compress && !full && !uncompressed_fits(L, dims)) return CPD_ERR_UNSUPPORTED;

  SolvePlan p; fill_dims(p, L, dims, R); p.dtype = dtype; p.full = full ? 1 : 0;
  Carver c(workspace, ws_bytes);
  plan_solve(p, c, o);
  if (!c.ok) return CPD_ERR_WORKSPACE;
  // ranks whose R x R Grams and Pi matrices alone exceed a CTA's shared memory
  if (!p.full && p.dgn_smem > smem_limit()) return CPD_ERR_UNSUPPORTED;
  if (p.rstate && p.r_smem > smem_limit()) return CPD_ERR_UNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  // replay a captured graph of the launch sequence when the stream allows it
  bool launched = false;
  int refine_loop = 0;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (st != nullptr && !profile_enabled() && cudaStreamIsCapturing(st, &cap) == cudaSuccess &&
      cap == cudaStreamCaptureStatusNone) {
    GraphKey k;
    memset(&k, 0, sizeof(k));
    cudaGetDevice(&k.dev);
    k.dtype = dtype; k.L = L; k.R = R;
    for (int l = 0; l < CPD_MAX_ORDER; ++l) k.dims[l] = p.dims[l];
    k.o = o; k.T = T; k.W0 = W0; k.W_out = W_out; k.lam = lambda_out; k.trace = trace;
    k.ws = workspace; k.ws_bytes = ws_bytes;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
    int loop = 0;
    {
      std::lock_guard<std::mutex> lk(g_graph_mu);
      for (auto& e : g_graphs)
        if (same_key(e.k, k)) {
          exec = e.exec; kernels = e.kernels; loop = e.refine_loop; e.used = ++g_graph_clock;
          break;
        }
    }
    if (exec == nullptr) {
      cudaGraph_t g = nullptr;
      cudaStream_t side = (o.refine_maxiter > 0 || full) ? side_stream() : nullptr;
      if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const long long before = cpd_launch_count();
        const int rc = enqueue_solve(p, o, T, dtype, L, R, W0, W_out, lambda_out, trace, st, side, &loop);
        kernels = cpd_launch_count() - before;
        count_launch(-(int)kernels);     // captured, not launched: counted when replayed
        const cudaError_t ec = cudaStreamEndCapture(st, &g);
        if (rc == CPD_OK && ec == cudaSuccess && g != nullptr &&
            cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
          std::lock_guard<std::mutex> lk(g_graph_mu);
          if (g_graphs.size() >= kMaxGraphs) {
            size_t victim = 0;
            for (size_t i = 1; i < g_graphs.size(); ++i)
              if (g_graphs[i].used < g_graphs[victim].used) victim = i;
            cudaGraphExecDestroy(g_graphs[victim].exec);
            g_graphs.erase(g_graphs.begin() + victim);
          }
          g_graphs.push_back(GraphEntry{k, exec, ++g_graph_clock, kernels, loop});
        } else {
          exec = nullptr;
          loop = 0;
        }
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();          // a failed capture falls back to direct launches
      }
    }
    if (exec != nullptr) {
      if (cudaGraphLaunch(exec, st) != cudaSuccess) return CPD_ERR_CUDA;
      count_launch((int)kernels);      // the kernels the graph replays (a loop body once)
      launched = true;
      refine_loop = loop;
    }
  }
  if (!launched) {
    const int rc = enqueue_solve(p, o, T, dtype, L, R, W0, W_out, lambda_out, trace, st);
    if (rc != CPD_OK) return rc;
  }

  if (info) {
    DevResult hr;
    int werr = 0;
    CK(cudaMemcpyAsync(&hr, p.res, sizeof(DevResult), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&werr, p.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    int core_dims[CPD_MAX_ORDER] = {0, 0, 0, 0};
    if (o.compress) CK(cudaMemcpyAsync(core_dims, p.core_dims_dev, sizeof(int) * CPD_MAX_ORDER, cudaMemcpyDeviceToHost, st));
    int r_iters = 0, r_stop = 0, r_cg = 0, r_status = CPD_OK, r_steps = 0; double r_err = 0.0, r_mu = 0.0;
    if (o.refine_maxiter > 0 || full)
      CK(read_refine_result(p.rstate, &r_iters, &r_stop, &r_cg, &r_err, &r_mu, &r_status, &r_steps, st));
    CK(cudaStreamSynchronize(st));
    // a replayed loop body ran max(0, steps - 1) times (the first step is
    // before the loop): correct the launch count by its 3 kernels a run
    if (refine_loop) count_launch(3 * ((r_steps > 1 ? r_steps - 1 : 0) - 1));
    memset(info, 0, sizeof(*info));
    info->status = hr.status;
    info->iters = hr.iters;
    info->stop_reason = hr.stop;
    info->cg_total = hr.cg_total;
    info->rel_err = hr.rel_err;
    info->mu = hr.mu;
    info->grad_inf = hr.grad_inf;
    for (int l = 0; l < L; ++l) info->core_dims[l] = o.compress ? core_dims[l] : p.idims[l];
    if (o.refine_maxiter > 0) {
      info->refine_iters = r_iters; info->refine_stop_reason = r_stop; info->refine_cg_total = r_cg;
      info->refine_rel_err = r_err; info->mu = r_mu;
      if (r_status != CPD_OK) info->status = r_status;
    }
    if (werr != 0) info->status = werr;        // a bounded device wait ran out
  }
  CK(cudaGetLastError());
  return CPD_OK;
}

int cpd_compress(const float* T, int L, const int64_t* dims, int R, const cpd_options* opts,
                 float* U_out, float* core_out, float* sigma_out, int* core_dims_out,
                 void* workspace, size_t ws_bytes, void* stream) {
  int v = validate_common(L, dims, R);
  if (v != CPD_OK) return v;
  if ((v = validate_options(opts)) != CPD_OK) return v;
  if (!T || !U_out || !core_out || !sigma_out || !workspace) return CPD_ERR_INVALID_ARG;
  cpd_options o; cpd_default_options(&o);
  if (opts) o = *opts;
  o.compress = 1; o.refine_maxiter = 0;
  if (o.gram_precision == CPD_GRAM_BF16 && !gram_bf16_tc_supported(dims[0], T)) return CPD_ERR_UNSUPPORTED;
  SolvePlan p; fill_dims(p, L, dims, R); p.dtype = CPD_F32;
  Carver c(workspace, ws_bytes);
  plan_solve(p, c, o);
  if (!c.ok) return CPD_ERR_WORKSPACE;
  // write straight into the caller's buffers
  p.U = U_out; p.sigma = sigma_out; p.core = core_out;
  cudaStream_t st = as_stream(stream);
  CK(cudaMemsetAsync(p.err, 0, sizeof(int), st));
  int rc = run_compress(p, T, o, st);
  if (rc != CPD_OK) return rc;
  if (core_dims_out) {
    int cd[CPD_MAX_ORDER];
    CK(cudaMemcpyAsync(cd, p.core_dims_dev, sizeof(int) * CPD_MAX_ORDER, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int l = 0; l < L; ++l) core_dims_out[l] = cd[l];
  }
  CK(cudaGetLastError());
  return CPD_OK;
}

int cpd_core_eval(const float* S, int L, const int64_t* dims, int R, const float* W,
                  float* f_out, float* g_out, double* fsq_out, void* workspace,
                  size_t ws_bytes, void* stream) {
  int v = validate_common(L, dims, R);
  if (v != CPD_OK) return v;
  if (!S || !W || !g_out || !fsq_out) return CPD_ERR_INVALID_ARG;
  int d[CPD_MAX_ORDER] = {1, 1, 1, 1};
  for (int l = 0; l < L; ++l) d[l] = (int)dims[l];
  CoreEvalArgs a{};
  a.R = R;
  for (int l = 0; l < CPD_MAX_ORDER; ++l) a.dims[l] = d[l];
  a.S = S; a.W = W; a.f_out = f_out; a.g_out = g_out; a.fsq_out = fsq_out;
  size_t sm = dgn_smem_bytes_host(L, d, R, 1);
  a.big_in_smem = sm <= smem_limit() ? 1 : 0;
  if (!a.big_in_smem) {
    sm = dgn_smem_bytes_host(L, d, R, 0);
    if (!workspace || ws_bytes < dgn_gscratch_floats_host(L, d, R) * 4) return CPD_ERR_WORKSPACE;
    a.gscratch = static_cast<float*>(workspace);
  }
  Shape s; make_shape(s, L, d, R);
  cudaStream_t st = as_stream(stream);
  PL("core_eval", launch_core_eval(L, a, 256, sm, st));
  return CPD_OK;
}

int cpd_jtj_apply(int L, const int64_t* dims, int R, const float* W, const float* V,
                  float* out, void* workspace, size_t ws_bytes, void* stream) {
  (void)workspace; (void)ws_bytes;
  int v = validate_common(L, dims, R);
  if (v != CPD_OK) return v;
  if (!W || !V || !out) return CPD_ERR_INVALID_ARG;
  int d[CPD_MAX_ORDER] = {1, 1, 1, 1};
  for (int l = 0; l < L; ++l) d[l] = (int)dims[l];
  JtjArgs a{};
  a.R = R;
  for (int l = 0; l < CPD_MAX_ORDER; ++l) a.dims[l] = d[l];
  a.W = W; a.V = V; a.out = out;
  size_t sm = dgn_smem_bytes_host(L, d, R, 0);
  if (sm > smem_limit()) return CPD_ERR_UNSUPPORTED;
  cudaStream_t st = as_stream(stream);
  PL("jtj_apply", launch_jtj_apply(L, a, 256, sm, st));
  return CPD_OK;
}

int cpd_mode_gram(const float* T, int L, const int64_t* dims, int mode, int precision,
                  float* G_out, void* workspace, size_t ws_bytes, void* stream) {
  int v = validate_common(L, dims, 1);
  if (v != CPD_OK) return v;
  if (!T || !G_out || mode < 0 || mode >= L) return CPD_ERR_INVALID_ARG;
  if (precision != CPD_GRAM_FP32 && precision != CPD_GRAM_BF16) return CPD_ERR_INVALID_ARG;
  if (precision == CPD_GRAM_BF16 && (mode != 0 || !gram_bf16_tc_supported(dims[0], T))) return CPD_ERR_UNSUPPORTED;
  long long a = 1, c = 1;
  for (int j = 0; j < mode; ++j) a *= dims[j];
  for (int j = mode + 1; j < L; ++j) c *= dims[j];
  cudaStream_t st = as_stream(stream);
  CK(cudaMemsetAsync(G_out, 0, sizeof(float) * (size_t)dims[mode] * dims[mode], st));
  if (precision == CPD_GRAM_BF16) {
    size_t need = gram_bf16_tc_scratch_bytes(dims[0], c);
    if (ws_bytes < need || (need > 0 && workspace == nullptr)) return CPD_ERR_WORKSPACE;
    PL("gram_bf16_tc", launch_gram_bf16_tc(T, dims[0], c, G_out, static_cast<float*>(workspace), ws_bytes, st));
  } else {
    View3 vv{a, dims[mode], c, nullptr, 0};
    PL("gram_fp32", launch_gram_simt(T, vv, a, G_out, st));
  }
  return CPD_OK;
}

int cpd_refine_eval(const float* T, int L, const int64_t* dims, int R, const float* W,
                    float* g_out, double* esq_out, void* workspace, size_t ws_bytes,
                    void* stream) {
  (void)workspace; (void)ws_bytes;
  int v = validate_common(L, dims, R);
  if (v != CPD_OK) return v;
  if (!T || !W || !g_out || !esq_out) return CPD_ERR_INVALID_ARG;
  if (!pass_ok(L, dims, R)) return CPD_ERR_UNSUPPORTED;
  RefinePassArgs pa{};
  pa.T = T; pa.L = L; pa.R = R; pa.W = W; pa.G = g_out; pa.esq = esq_out; pa.want_tsq = 1;
  for (int l = 0; l < CPD_MAX_ORDER; ++l) pa.dims[l] = (l < L) ? dims[l] : 1;
  pa.done = nullptr;
  cudaStream_t st = as_stream(stream);
  PL("refine_pass", launch_refine_pass(pa, st));
  return CPD_OK;
}

}  // extern "C"
