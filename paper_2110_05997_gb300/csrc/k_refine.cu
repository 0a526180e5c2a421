// dGN iterations on the full tensor after uncompression ("refinement"): each
// iteration is one pass over T (residual e = T - [[W]], ||e||^2 in FP64, the
// MTTKRP of e for every mode = -grad F; Sec. 4.1.3 formulas applied to T) and
// one single-CTA step (Grams, Pi, regulariser, PCG with Theorem "Hv",
// update, balance, gain ratio, damping and stop tests).
#include "kernels.h"
#include "solver.cuh"
#include "refine_pass.cuh"

namespace cpdk {

struct RefineState {
  double mu, F, normT, pred_drop, step;
  int kglob, cg_total, stop, status, iters, jnext;   // jnext: steps that got past the stop flag
  double rel_err;
};

size_t refine_state_bytes() { return sizeof(RefineState); }

__global__ void k_zero_pass(float* G, int n, double* esq, int want_tsq, const int* done) {
  if (done && *done) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) G[j] = 0.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) { esq[0] = 0.0; if (want_tsq) esq[1] = 0.0; }
}

// Supported shapes: I1 <= 256 * SLOTS with RMAX * SLOTS <= 64 (I1 <= 1024 for
// R <= 16, I1 <= 512 for R <= 32, I1 <= 256 for R <= 64), fibre indices below
// 2^31 and the pass's shared memory within one CTA's 227 KB.
bool refine_pass_supported(int L, const long long* dims, int R) {
  const long long I1 = dims[0];
  if (R <= 16 ? I1 > 1024 : R <= 32 ? I1 > 512 : I1 > 256) return false;
  long long nf = 1;
  for (int l = 1; l < L; ++l) nf *= dims[l];
  if (nf >= (1ll << 31)) return false;
  return pass_smem(L, dims, R) <= (size_t)227 * 1024;
}

cudaError_t launch_refine_pass(const RefinePassArgs& a, cudaStream_t st) {
  int n = 0;
  for (int l = 0; l < a.L; ++l) n += (int)a.dims[l] * a.R;
  if (!refine_pass_supported(a.L, a.dims, a.R)) return cudaErrorInvalidValue;
  k_zero_pass<<<16, 256, 0, st>>>(a.G, n, a.esq, a.want_tsq, a.done);
  count_launch();
  if (!a.cuda_cores && refine_tc_supported(a.L, a.dims, a.R, a.T)) return launch_refine_tc(a, st);
  const size_t smem = pass_smem(a.L, a.dims, a.R);
  long long nf = 1;
  for (int l = 1; l < a.L; ++l) nf *= a.dims[l];
  const long long nbatch = (nf + kNB - 1) / kNB;
  const int threads = a.dims[0] >= 256 ? 256 : (int)((a.dims[0] + 31) / 32 * 32);
  return a.L == 3 ? launch_refine_pass3(a, smem, threads, nbatch, st) : launch_refine_pass4(a, smem, threads, nbatch, st);
}

// ---- the single-CTA step ----------------------------------------------------------
size_t refine_step_smem_bytes(int L, const long long* dims, int R, int vec_in_smem, int blk) {
  size_t n = 0;
  for (int l = 0; l < L; ++l) n += (size_t)dims[l] * R;
  auto up = [](size_t x) { return (x + 3) & ~(size_t)3; };
  size_t f = small_buf_floats(L, R, blk);
  if (vec_in_smem) f += 7 * up(n);
  return 128 * sizeof(double) + f * sizeof(float);
}

// In a graph loop (use_cond) every exit sets the loop condition: 0 once the
// refinement has stopped or j = maxiter, else 1; j comes from the state's
// counter, so the body's launch arguments are the same in every iteration.
// RP > 0: ranks up to RP take the row-wise CG (pcg_rows), else pcg.
template <int L, int RP>
__global__ void __launch_bounds__(1024) k_refine_step(RefineStepArgs a) {
  if (*a.done) {
    if (a.use_cond && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0u);
    return;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_stop, s_j;
  __shared__ Shape s;
  if (threadIdx.x == 0) {
    int dims[kMaxL];
    for (int l = 0; l < kMaxL; ++l) dims[l] = (l < L) ? (int)a.dims[l] : 1;
    make_shape(s, L, dims, a.R);
    const int jj = a.j_from_state ? a.state->jnext : a.j;
    a.state->jnext = jj + 1;
    s_j = jj;
  }
  __syncthreads();
  const int jr = s_j;                          // this step's refinement iteration
  const int R = a.R;
  auto up = [](size_t x) { return (x + 3) & ~(size_t)3; };
  Bufs b{};
  b.red = reinterpret_cast<double*>(smem_raw);
  float* p = carve_small(b, reinterpret_cast<float*>(smem_raw + 128 * sizeof(double)), L, R, a.precond);
  float* vb = a.vec_in_smem ? p : a.vecs;
  float** vecs[7] = {&b.W, &b.G, &b.X, &b.Rr, &b.P, &b.Z, &b.Tmp};
  for (int v = 0; v < 7; ++v) { *vecs[v] = vb; vb += up((size_t)s.n); }
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) { b.W[j] = a.W[j]; b.G[j] = a.G[j]; }
  float gm = 0.f;
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) gm = fmaxf(gm, fabsf(a.G[j]));
  const double ginf = (double)block_max(gm, b.red);   // also a barrier
  RefineState* st = a.state;
  if (threadIdx.x == 0) {
    s_stop = 0;
    const double esq = a.esq[0];
    if (a.err && *a.err) {                      // the pass's bounded wait ran out: its sums are partial
      st->status = CPD_ERR_TIMEOUT;
      s_stop = 1;
    } else if (jr > a.maxiter) {                       // not reached: the loop condition ends at maxiter
      if (st->stop == CPD_STOP_NONE) st->stop = CPD_STOP_MAXITER;
      s_stop = 1;
    } else if (jr == 0) {
      st->normT = sqrt(a.esq[1]);
      st->F = 0.5 * esq;
      st->rel_err = st->normT > 0.0 ? sqrt(esq) / st->normT : 0.0;
      a.hist[0] = st->rel_err;
      if (!isfinite(esq)) { st->status = CPD_ERR_NUMERIC; s_stop = 1; }
    } else {
      double mu = st->mu;
      const double Fn = 0.5 * esq;
      const double gain = gain_update(st->F, Fn, st->pred_drop, mu, a.mu_min);
      const double e = st->normT > 0.0 ? quick_div(quick_sqrt(esq), st->normT) : 0.0;
      st->mu = mu; st->F = Fn; st->rel_err = e; st->iters = jr;
      a.hist[jr] = e;
      write_trace(a.trace, a.trace_cap, a.trace_slot0 + jr - 1, st->kglob, e, mu, gain,
                  -1, st->step, ginf, 1);
      int stop;
      if (!isfinite(esq) || !isfinite(st->step)) { st->status = CPD_ERR_NUMERIC; stop = CPD_STOP_NONE; s_stop = 1; }
      else {
        stop = stop_test(jr, a.maxiter, a.tol, e, st->step, ginf,
                         divergence_threshold(st->normT, a.tol), a.hist);
        if (stop != CPD_STOP_NONE) { st->stop = stop; s_stop = 1; }
      }
    }
    if (s_stop) *a.done = 1;
  }
  __syncthreads();
  if (s_stop) {
    if (a.use_cond && threadIdx.x == 0) cudaGraphSetConditional(a.cond, 0u);
    return;
  }
  const double mu = st->mu;
  __shared__ int s_maxit;
  const int kglob = st->kglob + 1;
  if (threadIdx.x == 0)
    s_maxit = (kglob <= a.cgtab_len) ? a.cgtab[kglob] : cg_maxiter(kglob, a.seed, a.cg_a, a.cg_b);
  grams_pi<L>(s, b);                           // its first barrier publishes s_maxit
  if (a.precond) regularize_block<L>(s, b, mu);
  else regularize<L>(s, b, mu);
  const int maxit = s_maxit;
  int its;
  if (a.precond) its = pcg_block<L>(s, b, mu, maxit, a.tol);
  else if constexpr (RP > 0) its = pcg_rows<L, RP>(s, b, mu, maxit, a.tol);
  else its = pcg<L>(s, b, mu, maxit, a.tol);
  double pred_drop, step;
  finish_step<L>(s, b, pred_drop, step);
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) a.W[j] = b.W[j];
  if (threadIdx.x == 0) {
    st->pred_drop = pred_drop; st->step = quick_sqrt(step); st->kglob = kglob; st->cg_total += its;
    if (a.trace && a.trace_slot0 + jr < a.trace_cap)
      a.trace[(size_t)(a.trace_slot0 + jr) * CPD_TRACE_FIELDS + 4] = its;
    if (a.use_cond) cudaGraphSetConditional(a.cond, jr + 1 <= a.maxiter ? 1u : 0u);
  }
}

template <int L, int RP>
cudaError_t launch_step_t(const RefineStepArgs& a, int threads, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_refine_step<L, RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_refine_step<L, RP><<<1, threads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_step_l(const RefineStepArgs& a, int threads, size_t smem, cudaStream_t st) {
  if (a.R <= 8) return launch_step_t<L, 8>(a, threads, smem, st);
  if (a.R <= 12) return launch_step_t<L, 12>(a, threads, smem, st);
  if (a.R <= 16) return launch_step_t<L, 16>(a, threads, smem, st);
  return launch_step_t<L, 0>(a, threads, smem, st);
}

cudaError_t launch_refine_step(const RefineStepArgs& a, int threads, size_t smem, cudaStream_t st) {
  return a.L == 3 ? launch_step_l<3>(a, threads, smem, st) : launch_step_l<4>(a, threads, smem, st);
}

__global__ void k_refine_init(RefineState* s, const DevResult* core, int* done) {
  s->mu = core->mu; s->F = 0.0; s->normT = 0.0; s->pred_drop = 0.0; s->step = 0.0;
  s->kglob = core->kglob; s->cg_total = 0; s->stop = 0; s->status = CPD_OK; s->iters = 0; s->jnext = 0;
  s->rel_err = 0.0;
  *done = (core->status != CPD_OK) ? 1 : 0;
}

cudaError_t launch_refine_init(RefineState* state, const DevResult* core_res, int* done, cudaStream_t st) {
  k_refine_init<<<1, 1, 0, st>>>(state, core_res, done);
  count_launch();
  return cudaGetLastError();
}

cudaError_t read_refine_result(const RefineState* state, int* iters, int* stop, int* cg_total,
                               double* rel_err, double* mu, int* status, int* steps_run, cudaStream_t st) {
  static thread_local RefineState h;
  cudaError_t e = cudaMemcpyAsync(&h, state, sizeof(RefineState), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  *iters = h.iters; *stop = h.stop; *cg_total = h.cg_total; *rel_err = h.rel_err; *mu = h.mu;
  *status = h.status;
  if (steps_run) *steps_run = h.jnext;
  return cudaSuccess;
}

}  // namespace cpdk

// ---- dGN on a large tensor without compression: every iteration a pass ----------
namespace cpdk {

__global__ void k_abs_sum(const float* T, long long N, double* out) {
  float acc = 0.f;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x)
    acc += fabsf(T[e]);
  __shared__ double red[32];
  double d = (double)acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x < 32) {
    d = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (threadIdx.x == 0) atomicAdd(out, d);
  }
}

// The starting factors on the full tensor (Sec. 4.1.2: random N(0,1) draws of
// the same SplitMix64 stream as the core solver, or the caller's), balanced
// (Sec. 4.1.3 "Updates"), mu0 = tau mean|T| (Sec. 4.1.3) into the record the
// refinement state is primed from, and the table of CG iteration caps (the
// core solver's prologue fills it on the compressed path).
__global__ void __launch_bounds__(1024) k_full_start(int L, Dims4 dims, int R, int init, const float* W0,
                                                     uint64_t seed, double tau, const double* abs_sum, float* W,
                                                     DevResult* res, int* cgtab, int cgtab_len, double cg_a,
                                                     double cg_b) {
  fill_cg_table(cgtab, cgtab_len, seed, cg_a, cg_b);
  long long off[CPD_MAX_ORDER + 1];
  off[0] = 0;
  long long N = 1;
  for (int l = 0; l < L; ++l) { off[l + 1] = off[l] + dims.v[l] * R; N *= dims.v[l]; }
  const long long n = off[L];
  for (long long j = threadIdx.x; j < n; j += blockDim.x)
    W[j] = init == CPD_INIT_GIVEN ? W0[j] : (float)normal_draw(seed, (uint64_t)j);
  __syncthreads();
  __shared__ float nrm[CPD_MAX_ORDER * CPD_MAX_RANK];
  for (int q = threadIdx.x; q < L * R; q += blockDim.x) {
    const int l = q / R, r = q - l * R;
    const float* w = W + off[l] + (long long)r * dims.v[l];
    float acc = 0.f;
    for (long long i = 0; i < dims.v[l]; ++i) acc = fmaf(w[i], w[i], acc);
    nrm[q] = sqrtf(acc);
  }
  __syncthreads();
  __shared__ float scl[CPD_MAX_ORDER * CPD_MAX_RANK];
  for (int q = threadIdx.x; q < L * R; q += blockDim.x) {
    const int l = q / R, r = q - l * R;
    float lg = 0.f;
    bool ok = true;
    for (int j = 0; j < L; ++j) { const float v = nrm[j * R + r]; ok = ok && v > 0.f; lg += ok ? logf(v) : 0.f; }
    scl[q] = ok ? expf(lg / L) / nrm[q] : 1.f;
  }
  __syncthreads();
  for (int l = 0; l < L; ++l)
    for (long long j = threadIdx.x; j < dims.v[l] * R; j += blockDim.x) W[off[l] + j] *= scl[l * R + j / dims.v[l]];
  if (threadIdx.x == 0) {
    res->status = CPD_OK; res->iters = 0; res->stop = 0; res->cg_total = 0; res->kglob = 0; res->pad0 = 0;
    res->mu = tau * (*abs_sum) / (double)N;
    res->rel_err = 0.0; res->grad_inf = 0.0; res->normS = 0.0;
  }
}

cudaError_t launch_full_start(int L, const long long* dims, int R, int init, const float* W0, uint64_t seed,
                              double tau, const float* T, double* abs_sum, float* W, DevResult* res, int* cgtab,
                              int cgtab_len, double cg_a, double cg_b, cudaStream_t st) {
  long long N = 1;
  Dims4 d{};
  for (int l = 0; l < CPD_MAX_ORDER; ++l) d.v[l] = l < L ? dims[l] : 1;
  for (int l = 0; l < L; ++l) N *= dims[l];
  cudaError_t e = cudaMemsetAsync(abs_sum, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_abs_sum<<<4 * sms, 512, 0, st>>>(T, N, abs_sum);
  count_launch();
  k_full_start<<<1, 1024, 0, st>>>(L, d, R, init, W0, seed, tau, abs_sum, W, res, cgtab, cgtab_len, cg_a, cg_b);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cpdk

namespace cpdk {

// The outcome of a run of pass-based iterations as the solve's result record
// (dGN on T without compression: the iterations are the solve).
__global__ void k_refine_result(const RefineState* s, DevResult* r) {
  r->status = s->status; r->iters = s->iters; r->stop = s->stop; r->cg_total = s->cg_total;
  r->kglob = s->kglob; r->pad0 = 0;
  r->rel_err = s->rel_err; r->mu = s->mu; r->grad_inf = 0.0; r->normS = s->normT;
}

cudaError_t launch_refine_result(const RefineState* state, DevResult* res, cudaStream_t st) {
  k_refine_result<<<1, 1, 0, st>>>(state, res);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cpdk
