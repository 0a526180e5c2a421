// The single-CTA damped Gauss-Newton solve (Sec. 4.1.3) as a device function:
// load the tensor, initialise (Sec. 4.1.2), balance, iterate (Grams and Pi,
// regulariser and preconditioner, PCG with Theorem "Hv", update, balance,
// residual and MTTKRP gradient, gain ratio, damping, stop tests) and write
// the balanced factors and the outcome.  Used by the single-tensor kernel and
// by the batched solver (one CTA per CPD).
#pragma once

#include "kernels.h"
#include "solver.cuh"

namespace cpdk {

// big_in_smem: 1 = every buffer in shared memory; 0 = the tensor-sized ones in
// the global scratch; -1 = the seven solver vectors there too (high ranks,
// whose R x R Grams and Pi matrices leave no room for them).
__host__ __device__ inline size_t dgn_smem_bytes(int L, const int* d, int R, int big_in_smem, int blk = 0) {
  Shape s; make_shape(s, L, d, R);
  size_t f = 0;
  auto up = [](size_t x) { return (x + 3) & ~(size_t)3; };   // 16-byte granules
  f += small_buf_floats(L, R, blk);
  if (big_in_smem >= 0) f += 7 * up((size_t)s.n);
  if (big_in_smem > 0) {
    const size_t NL = s.N / s.d[L - 1], N0 = s.N / s.d[0];
    f += 2 * up((size_t)s.N) + up(R * NL) + up(R * N0);
  }
  return 128 * sizeof(double) + f * sizeof(float);
}

__host__ __device__ inline size_t dgn_gscratch_floats(int L, const int* d, int R, int big_in_smem = 0) {
  Shape s; make_shape(s, L, d, R);
  const size_t NL = s.N / s.d[L - 1], N0 = s.N / s.d[0];
  auto up = [](size_t x) { return (x + 63) & ~(size_t)63; };
  return (big_in_smem < 0 ? 7 * up((size_t)s.n) : 0) + 2 * up((size_t)s.N) + up(R * NL) + up(R * N0);
}

// Carve the solver's buffers: small ones always in shared memory, the vectors
// there unless big_in_smem < 0, tensor-sized ones there when big_in_smem > 0;
// the rest in the global scratch (layout of dgn_gscratch_floats).
__device__ inline void carve(const Shape& s, Bufs& b, unsigned char* smem, float* gscratch,
                      int big_in_smem, float** Sbuf, int blk = 0) {
  const int L = s.L, R = s.R;
  auto up = [](size_t x) { return (x + 3) & ~(size_t)3; };
  auto up64 = [](size_t x) { return (x + 63) & ~(size_t)63; };
  b.red = reinterpret_cast<double*>(smem);
  float* p = carve_small(b, reinterpret_cast<float*>(smem + 128 * sizeof(double)), L, R, blk);
  float* gq = gscratch;
  float** vecs[7] = {&b.W, &b.G, &b.X, &b.Rr, &b.P, &b.Z, &b.Tmp};
  for (int v = 0; v < 7; ++v) {
    if (big_in_smem >= 0) { *vecs[v] = p; p += up((size_t)s.n); }
    else { *vecs[v] = gq; gq += up64((size_t)s.n); }
  }
  const size_t NL = s.N / s.d[L - 1], N0 = s.N / s.d[0];
  float* q = p;
  size_t a16 = 4;
  if (big_in_smem <= 0) { q = gq; a16 = 64; }
  auto upg = [a16](size_t x) { return (x + a16 - 1) & ~(a16 - 1); };
  *Sbuf = q; q += upg((size_t)s.N);
  b.F = q; q += upg((size_t)s.N);
  b.Kb = q; q += upg(R * NL);
  b.Bb = q; q += upg(R * N0);
  b.S = *Sbuf;
}

// Load the tensor into the solver's buffer (FP64 input is rounded to FP32),
// and return ||S|| and mean|S| (FP64 accumulation).
__device__ inline void load_tensor(const Shape& s, const void* src, int f64, float* dst, double* red,
                            double& norm, double& meanabs) {
  float vf[2] = {0.f, 0.f};
  for (int e = threadIdx.x; e < s.N; e += blockDim.x) {
    const float x = f64 ? (float)static_cast<const double*>(src)[e] : static_cast<const float*>(src)[e];
    dst[e] = x;
    vf[0] = fmaf(x, x, vf[0]);
    vf[1] += fabsf(x);
  }
  double v[2];
  block_sum<2>(vf, v, red);
  norm = sqrt(v[0]);
  meanabs = v[1] / (double)s.N;
}

// Initialisation (Sec. 4.1.2).  MLSVD-energy: the R entries of largest |s|
// (ties to the smaller column-major index) as rank-one terms s e_j1 o ... o e_jL,
// s on mode 1.  Random: N(0,1) by Box-Muller on SplitMix64.  Given: copy.
template <int L>
__device__ void init_factors(const Shape& s, const Bufs& b, int mode, const float* W0,
                             uint64_t seed, int* chosen) {
  const int R = s.R;
  if (mode == CPD_INIT_GIVEN) {
    for (int j = threadIdx.x; j < s.n; j += blockDim.x) b.W[j] = W0[j];
  } else if (mode == CPD_INIT_RANDOM) {
    for (int j = threadIdx.x; j < s.n; j += blockDim.x) b.W[j] = (float)normal_draw(seed, (uint64_t)j);
  } else {
    for (int j = threadIdx.x; j < s.n; j += blockDim.x) b.W[j] = 0.f;
    const int take = R < s.N ? R : s.N;
    for (int r = 0; r < take; ++r) {
      float best = -1.f; int bi = 0x7fffffff;
      for (int e = threadIdx.x; e < s.N; e += blockDim.x) {
        bool used = false;
        for (int t = 0; t < r; ++t) used |= (chosen[t] == e);
        float v = fabsf(b.S[e]);
        if (!(v == v)) v = -0.5f;              // a NaN entry is still a valid choice
        if (!used && (v > best || (v == best && e < bi))) { best = v; bi = e; }
      }
      block_argmax(best, bi, b.red);
      if (threadIdx.x == 0) chosen[r] = bi;
      __syncthreads();
    }
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
      int e = chosen[r % take];
      const float val = b.S[e];
#pragma unroll
      for (int l = 0; l < L; ++l) {
        const int il = e % s.d[l]; e /= s.d[l];
        b.W[s.off[l] + r * s.d[l] + il] = (l == 0) ? val : 1.f;
      }
    }
  }
  __syncthreads();
}

template <int L>
__device__ void dgn_run(const DgnArgs& a, unsigned char* smem_raw) {
  __shared__ State st;
  __shared__ int chosen[kMaxR];
  __shared__ Shape s;       // shared: indexed by runtime mode numbers in every phase
  if (threadIdx.x == 0) {
    int dims[kMaxL];
    for (int l = 0; l < kMaxL; ++l) dims[l] = (l < L) ? (a.dev_dims ? a.dev_dims[l] : a.dims[l]) : 1;
    make_shape(s, L, dims, a.R);
  }
  __syncthreads();
  Bufs b; float* Sbuf;
  carve(s, b, smem_raw, a.gscratch, a.big_in_smem, &Sbuf, a.precond);

  double normS, meanabs;
  load_tensor(s, a.S, a.s_f64, Sbuf, b.red, normS, meanabs);
  fill_cg_table(a.cgtab, a.cgtab_len, a.seed, a.cg_a, a.cg_b);
  double fsq, ginf;
  __shared__ int s_init_used;
  if (a.init == CPD_INIT_LEARNED) {
    // two candidate starts: the MLSVD-energy start and the network's factors
    // (a.W0); dGN starts from the network's only when its residual is below
    // half the MLSVD start's (norms; a smaller margin let starts from worse
    // basins through and cost iterations on the 16^3 workload); the MLSVD
    // start is the fallback.  a.W_out holds the first candidate meanwhile.
    init_factors<L>(s, b, CPD_INIT_MLSVD, nullptr, a.seed, chosen);
    balance<L>(s, b);
    double f_mlsvd, g_mlsvd;
    core_pass<L>(s, b, f_mlsvd, g_mlsvd);
    for (int j = threadIdx.x; j < s.n; j += blockDim.x) a.W_out[j] = b.W[j];
    init_factors<L>(s, b, CPD_INIT_GIVEN, a.W0, a.seed, chosen);
    balance<L>(s, b);
    core_pass<L>(s, b, fsq, ginf);
    if (threadIdx.x == 0) s_init_used = (isfinite(fsq) && fsq < 0.25 * f_mlsvd) ? 1 : 0;
    __syncthreads();
    if (!s_init_used) {
      for (int j = threadIdx.x; j < s.n; j += blockDim.x) b.W[j] = a.W_out[j];
      __syncthreads();
      core_pass<L>(s, b, fsq, ginf);
    }
  } else {
    init_factors<L>(s, b, a.init, a.W0, a.seed, chosen);
    balance<L>(s, b);
    core_pass<L>(s, b, fsq, ginf);
    if (threadIdx.x == 0) s_init_used = 0;
  }
  if (threadIdx.x == 0) {
    st.mu = a.mu0 >= 0.0 ? a.mu0 : a.tau * meanabs;
    st.F = 0.5 * fsq;
    st.normS = normS;
    st.rel_err = normS > 0.0 ? sqrt(fsq) / normS : 0.0;
    st.grad_inf = ginf;
    st.kglob = a.k0; st.cg_total = 0; st.stop = 0; st.iters = 0;
    st.status = isfinite(fsq) ? CPD_OK : CPD_ERR_NUMERIC;
    if (st.status != CPD_OK) st.stop = CPD_STOP_NONE;
    a.hist[0] = st.rel_err;
  }
  __shared__ double s_div;
  if (threadIdx.x == 0) s_div = divergence_threshold(st.normS, a.tol);
  __syncthreads();
  const bool bad0 = st.status != CPD_OK;
  __shared__ int s_maxit;
  for (int k = 1; k <= a.maxiter && !bad0; ++k) {
    const double mu = st.mu;
    if (threadIdx.x == 0)
      s_maxit = (a.k0 + k <= a.cgtab_len) ? a.cgtab[a.k0 + k] : cg_maxiter(a.k0 + k, a.seed, a.cg_a, a.cg_b);
    grams_pi<L>(s, b);                         // its first barrier publishes s_maxit
    if (a.precond) regularize_block<L>(s, b, mu);
    else regularize<L>(s, b, mu);
    const int maxit = s_maxit;
    const int its = a.precond ? pcg_block<L>(s, b, mu, maxit, a.tol)
                    : (s.n <= (int)blockDim.x) ? pcg_owned<L>(s, b, mu, maxit, a.tol) : pcg<L>(s, b, mu, maxit, a.tol);
    double pred_drop, step;
    finish_step<L>(s, b, pred_drop, step);
    core_pass<L>(s, b, fsq, ginf);
    if (threadIdx.x == 0) {
      step = quick_sqrt(step);
      double m = st.mu;
      const double Fn = 0.5 * fsq;
      const double gain = gain_update(st.F, Fn, pred_drop, m, a.mu_min);
      const double e = st.normS > 0.0 ? quick_div(quick_sqrt(fsq), st.normS) : 0.0;
      st.mu = m; st.F = Fn; st.rel_err = e; st.grad_inf = ginf;
      st.cg_total += its; st.iters = k; st.kglob = a.k0 + k;
      a.hist[k] = e;
      write_trace(a.trace, a.trace_cap, a.trace_slot0 + k - 1, a.k0 + k, e, m, gain, its, step,
                  ginf, 0);
      if (!isfinite(fsq) || !isfinite(step)) { st.status = CPD_ERR_NUMERIC; st.stop = CPD_STOP_NONE; }
      else st.stop = stop_test(k, a.maxiter, a.tol, e, step, ginf, s_div, a.hist);
    }
    __syncthreads();
    if (st.stop != CPD_STOP_NONE || st.status != CPD_OK) break;
  }
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) a.W_out[j] = b.W[j];
  if (threadIdx.x == 0) {
    DevResult* r = a.res;
    r->status = st.status; r->iters = st.iters; r->stop = st.stop; r->cg_total = st.cg_total;
    r->kglob = st.kglob; r->rel_err = st.rel_err; r->mu = st.mu; r->grad_inf = st.grad_inf;
    r->pad0 = s_init_used;                     // 1: started from the learned factors
    r->normS = st.normS;
  }
}

}  // namespace cpdk
