// Argument blocks and host-side launchers of the CPD kernels (internal header
// shared by the translation units of libcpd).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/cpd.h"

namespace cpdk {

struct DevResult;

struct Dims4 { long long v[CPD_MAX_ORDER]; };

// Diagnostics (diag.cu): every kernel launch is counted; while profiling is
// enabled a ProfScope records a CUDA event pair around its launches.
void count_launch(int n = 1);
bool profile_enabled();
struct ProfScope {
  ProfScope(cudaStream_t st, const char* name);
  ~ProfScope();
  cudaStream_t st_; const char* name_; cudaEvent_t a_;
};

// Single-CTA dGN on an in-CTA tensor (k_dgn.cu).
struct DgnArgs {
  int R;
  int dims[CPD_MAX_ORDER];
  const int* dev_dims;        // core dims decided on the device, or nullptr
  const void* S;              // tensor (global), FP32 or FP64
  int s_f64;
  const float* W0;            // INIT_GIVEN factors (core space) or nullptr
  int init;
  uint64_t seed;
  double tol, tau, cg_a, cg_b;
  int maxiter;
  double mu0;                 // < 0: tau * mean|S|
  double mu_min;              // floor of mu after each update (0: none)
  int precond;                // 0: diagonal (Jacobi) preconditioner; 1: block-Jacobi
  int k0;                     // global iteration offset for cg_maxiter
  int big_in_smem;
  float* gscratch;            // tensor-sized buffers when not in shared memory
  double* hist;               // maxiter + 1 doubles
  double* trace;              // CPD_TRACE_FIELDS doubles per record, or nullptr
  int trace_cap, trace_slot0;
  float* W_out;               // balanced factors, stacked blocks
  DevResult* res;
  int* cgtab;                 // cg_maxiter(k) for k = 1..cgtab_len, filled in the prologue
  int cgtab_len;
};

struct CoreEvalArgs {
  int R;
  int dims[CPD_MAX_ORDER];
  const float* S;
  const float* W;
  float* f_out;
  float* g_out;
  double* fsq_out;
  int big_in_smem;
  float* gscratch;
};

struct JtjArgs {
  int R;
  int dims[CPD_MAX_ORDER];
  const float* W;
  const float* V;
  float* out;
};

size_t dgn_smem_bytes_host(int L, const int* d, int R, int big_in_smem, int blk = 0);

// CTA size of the single-CTA solvers: one thread per unknown, rounded up to
// whole warps (every per-entry phase of the CG then takes one pass; more
// warps than that only add barrier cost), at least 4 warps, at most 1024.
inline int threads_for(const cpd_options* o, int n) {
  if (o && o->block_threads > 0) return o->block_threads;
  int t = (n + 31) / 32 * 32;
  if (t < 128) t = 128;
  if (t > 1024) t = 1024;
  return t;
}
size_t dgn_gscratch_floats_host(int L, const int* d, int R, int big_in_smem = 0);

cudaError_t launch_dgn_core(int L, const DgnArgs& a, int threads, size_t smem, cudaStream_t st);
// The same solve by a cluster of csize CTAs (k_dgn_cluster.cu) for cores too
// large for one CTA's shared memory: FP32 tensor, each CTA a slice of fibres.
size_t dgn_cluster_smem_bytes_host(int L, const int* d, int R, int csize, int blk = 0);
cudaError_t launch_dgn_cluster(int L, const DgnArgs& a, int threads, int csize, size_t smem, cudaStream_t st);
cudaError_t launch_core_eval(int L, const CoreEvalArgs& a, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_jtj_apply(int L, const JtjArgs& a, int threads, size_t smem, cudaStream_t st);

// ---- compression (k_compress.cu) ---------------------------------------------
// A tensor viewed as (a, b, c) around mode l: a = prod_{j<l} dims, b = dims[l],
// c = prod_{j>l} dims.  Under ST-MLSVD, `a` depends on truncation ranks decided
// on the device: a = a_host * prod(dev_ranks[0..nr-1]) when dev_ranks != nullptr.
struct View3 {
  long long a_host, b, c;
  const int* dev_ranks;       // ranks of the modes before l (device), or nullptr
  int nr;
};

cudaError_t launch_gram_simt(const float* T, View3 v, long long a_max, float* G, cudaStream_t st);
// err / budget: see RefinePassArgs (a pipeline wait that runs out sets *err)
cudaError_t launch_gram_bf16_tc(const float* T, long long I, long long C, float* G, float* scratch,
                                size_t scratch_bytes, cudaStream_t st, int* err = nullptr, long long budget = 0);
size_t gram_bf16_tc_scratch_bytes(long long I, long long C);
bool gram_bf16_tc_supported(long long I, const float* T);
// D(m, n) = epilogue(sum_k A(m, k) B(n, k)) on BF16 tensor cores (FP32 operands
// rounded on load, FP32 accumulation); A(m, k) = A[m sam + k sak],
// B(n, k) = B[n sbn + k sbk]; epilogue: + bias[n], ReLU, x [mask(m, n) > 0],
// D[m ldd + n] = or += (accumulate).
struct GemmArgs {
  const float* A; long long sam, sak;
  const float* B; long long sbn, sbk;
  float* D; long long ldd;
  const float* bias;
  const float* mask; long long ldm;
  int M, N, K, relu, accumulate;
};
cudaError_t launch_gemm_tc(const GemmArgs& a, cudaStream_t st);

struct EigArgs {
  const float* G;             // I x I
  int I, P;                   // P = min(I, R) leading eigenpairs
  float* U;                   // I x P, column-major
  float* sigma;               // P
  int* rank_out;              // device: truncation rank of this mode
  double mlsvd_tol;
  int L;
  uint64_t seed;
  float* work;                // global scratch when G does not fit shared memory
  int fp32_only;              // 1: no FP64 polishing (the Gram itself is BF16-rounded)
};
cudaError_t launch_eig(const EigArgs& a, cudaStream_t st);
size_t eig_work_floats(int I, int P);
// Y(a, r, c) = sum_j U[j, r] T(a, j, c), r < rank (device) <= rmax.  The first
// mode (a = 1) runs on tensor cores when project_tc_supported (err / budget:
// see RefinePassArgs).
cudaError_t launch_project(const float* T, View3 v, long long a_max, const float* U,
                           const int* dev_rank, int rmax, float* Y, cudaStream_t st,
                           int* err = nullptr, long long budget = 0);
// First-mode projection on TF32 tensor cores with the three-product split
// (k_project_tc.cu): 32 <= I <= 256, I % 4 == 0, c >= 128, rmax <= 16, T 16-byte aligned.
bool project_tc_supported(long long I, long long c, int rmax, const float* T);
cudaError_t launch_project_tc(const float* T, long long I, long long c, const float* U, const int* dev_rank,
                              int rmax, float* Y, cudaStream_t st, int* err = nullptr, long long budget = 0);
// Pack the truncated core (dims from the device) from a buffer laid out with
// the same truncated dims: a copy (kept separate for clarity of ownership).
cudaError_t launch_copy_f32(const float* src, float* dst, long long n, cudaStream_t st);

// ---- uncompression, refinement, output (k_refine.cu) -----------------------------
struct PlanDims {                 // device-side dims of the current problem
  int core[CPD_MAX_ORDER];
};
cudaError_t launch_uncompress(int L, const long long* dims, int R, const float* U, const int* core_dims,
                              const int* Pdims, const float* Wc, float* Wfull, cudaStream_t st);
cudaError_t launch_project_given(int L, const long long* dims, int R, const float* U,
                                 const int* core_dims, const int* Pdims, const float* W0,
                                 float* Wc, cudaStream_t st);
cudaError_t launch_normalize(int L, const long long* dims, int R, const float* W, float* W_out,
                             float* lam_out, cudaStream_t st);

struct RefineState;
struct RefinePassArgs {
  const float* T;
  long long dims[CPD_MAX_ORDER];
  int L, R;
  const float* W;             // stacked factors (global)
  float* G;                   // stacked MTTKRP of the residual (zeroed by the launcher)
  double* esq;                // [0] = ||e||^2, [1] = ||T||^2 (if want_tsq)
  int want_tsq;
  const int* done;            // skip when *done != 0 (refinement stopped)
  int* err;                   // set to CPD_ERR_TIMEOUT by a bounded wait that ran out (or nullptr)
  long long budget;           // bound of every wait in SM clock cycles (0 = default)
  int cuda_cores;             // 1: force the CUDA-core pass
};
cudaError_t launch_refine_pass(const RefinePassArgs& a, cudaStream_t st);
bool refine_pass_supported(int L, const long long* dims, int R);
// the tensor-core pass (k_refine_tc.cu): R <= 16, I1 % 4 == 0, I1 <= 256,
// T 16-byte aligned, fewer than 2^31 fibres, its shared memory within 227 KB
bool refine_tc_supported(int L, const long long* dims, int R, const float* T);
cudaError_t launch_refine_tc(const RefinePassArgs& a, cudaStream_t st);

struct RefineStepArgs {
  int L, R;
  long long dims[CPD_MAX_ORDER];
  float* W;                   // global stacked factors (updated in place)
  const float* G;             // global MTTKRP of the residual at W
  const double* esq;          // ||e||^2 at W, ||T||^2
  RefineState* state;         // global
  float* vecs;                // global scratch for the CG vectors if not in shared memory
  int vec_in_smem;
  int j;                      // refinement iteration index (0 = only prime the state)
  int maxiter;
  double tol, cg_a, cg_b;
  double mu_min;              // floor of mu after each update (0: none)
  uint64_t seed;
  double* hist;               // maxiter + 1
  double* trace;
  int trace_cap, trace_slot0;
  int* done;
  const int* cgtab;           // cg_maxiter(k) table written by the core solver
  int cgtab_len;
  int j_from_state;           // 1: j is the state's iteration counter (a graph loop body)
  int use_cond;               // 1: set `cond` to 1 when another iteration follows, else 0
  cudaGraphConditionalHandle cond;
  const int* err;             // nonzero: a bounded wait of the pass ran out; the refinement stops
  int precond;                // 0: diagonal (Jacobi) preconditioner; 1: block-Jacobi
};
size_t refine_step_smem_bytes(int L, const long long* dims, int R, int vec_in_smem, int blk = 0);
cudaError_t launch_refine_step(const RefineStepArgs& a, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_refine_init(RefineState* state, const DevResult* core_res, int* done,
                               cudaStream_t st);
// The state after a run of pass-based iterations as the solve's result record.
cudaError_t launch_refine_result(const RefineState* state, DevResult* res, cudaStream_t st);
// dGN on a large tensor without compression (every iteration a pass over T):
// the balanced starting factors on T (random or given) into W and mu0 =
// tau mean|T| into *res, from which launch_refine_init primes the state.
cudaError_t launch_full_start(int L, const long long* dims, int R, int init, const float* W0, uint64_t seed,
                              double tau, const float* T, double* abs_sum, float* W, DevResult* res, int* cgtab,
                              int cgtab_len, double cg_a, double cg_b, cudaStream_t st);
size_t refine_state_bytes();
cudaError_t read_refine_result(const RefineState* state, int* iters, int* stop, int* cg_total,
                               double* rel_err, double* mu, int* status, int* steps_run, cudaStream_t st);

// ---- batched (k_batch.cu) ----------------------------------------------------------
struct BatchItem {
  long long t_off, w_off, l_off;
  int d[3];
  int R;
  int b;                      // index of the item in the caller's order
  int pad;
};
struct BatchArgs {
  const float* T;
  float* W;
  float* lam;
  const BatchItem* items;     // device, sorted longest-first
  int B;
  int* queue;                 // device work counter (zeroed by the launcher)
  cpd_info* infos;            // device
  float* scratch;             // per-CTA scratch
  size_t scratch_floats_per_cta;
  double* hist;               // per-CTA history, maxiter + 1 each
  int maxiter;
  double tol, tau, cg_a, cg_b, mlsvd_tol;
  double mu_min;              // floor of mu after each update (0: none)
  int compress, init;
  uint64_t seed;
  int ctas;
  // phased runs around the learned initialiser (0 = the whole method in one pass)
  int phase;                  // 1: compress and store; 2: solve from the store
  float* store;               // per-item store, store_floats each (caller's order)
  size_t store_floats;
  float* X;                   // phase 1: network input rows (B x CPD_INITNET_IN_PAD) or null
  const float* Y;             // phase 2: network outputs (B x CPD_INITNET_OUT) for CPD_INIT_LEARNED
  float* target;              // phase 2: training targets (B x CPD_INITNET_OUT) or null
  float* tmask;               // phase 2: their masks or null
};
size_t batch_smem_bytes(int dmax, int Rmax, int compress);
size_t batch_store_floats(int dmax, int Rmax);
// learned initialiser network (initnet.cu)
size_t initnet_param_count();
size_t initnet_act_bytes(int B);
cudaError_t initnet_forward(const float* P, const float* X, int B, void* ws, float* y, cudaStream_t st);
cudaError_t initnet_grad(const float* P, const float* X, const float* t, const float* mask, int B, void* ws,
                         float* G, double* loss_out, cudaStream_t st);
cudaError_t initnet_adam(float* P, float* m, float* v, const float* G, int step, double lr, double b1, double b2,
                         double eps, cudaStream_t st);
size_t batch_scratch_floats(int dmax, int Rmax);
cudaError_t launch_batch(const BatchArgs& a, int threads, size_t smem, cudaStream_t st);

}  // namespace cpdk
