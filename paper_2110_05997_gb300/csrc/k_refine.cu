// dGN iterations on the full tensor after uncompression ("refinement"): each
// iteration is one pass over T (residual e = T - [[W]], ||e||^2 in FP64, the
// MTTKRP of e for every mode = -grad F; Sec. 4.1.3 formulas applied to T) and
// one single-CTA step (Grams, Pi, regulariser, PCG with Theorem "Hv",
// update, balance, gain ratio, damping and stop tests).
#include "kernels.h"
#include "solver.cuh"

namespace cpdk {

struct RefineState {
  double mu, F, normT, pred_drop, step;
  int kglob, cg_total, stop, status, iters, pad;
  double rel_err;
};

size_t refine_state_bytes() { return sizeof(RefineState); }

// ---- the pass over T --------------------------------------------------------------
// Mode-1 fibers (I1 contiguous floats) in batches of kNB: for fiber f with
// kr_r = prod_{l>=2} W_l[i_l, r]:  t~ = sum_r W1[i1, r] kr_r, e = t - t~;
// G1 += E KR (register accumulators per thread); q = E^T W1 per fiber, then
// G_l[i_l, r] += q_r prod_{j>=2, j!=l} W_j[i_j, r] (shared atomics).
constexpr int kNB = 32;
constexpr int kPassThreads = 256;
constexpr int kG1Reg = 16;

template <int L>
__global__ void __launch_bounds__(kPassThreads) k_refine_pass(RefinePassArgs a) {
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) float sm[];
  const int R = a.R;
  const int I1 = (int)a.dims[0];
  int d[kMaxL], off[kMaxL + 1];
  off[0] = 0;
#pragma unroll
  for (int l = 0; l < kMaxL; ++l) d[l] = (l < L) ? (int)a.dims[l] : 1;
#pragma unroll
  for (int l = 0; l < L; ++l) off[l + 1] = off[l] + d[l] * R;
  const int n = off[L];
  long long nf = 1;
#pragma unroll
  for (int l = 1; l < L; ++l) nf *= d[l];
  // shared: W (n) | Gs for modes >= 2 (n - I1*R, indexed from off[1]) | E (I1 x (kNB+1)) | KR (kNB x R) | Q (kNB x R)
  float* Ws = sm;
  float* Gs = Ws + n;                // entries [off[1], n) used
  float* E = Gs + n;
  float* KR = E + (size_t)I1 * (kNB + 1);
  float* Qs = KR + kNB * R;
  for (int j = threadIdx.x; j < n; j += blockDim.x) { Ws[j] = a.W[j]; Gs[j] = 0.f; }
  __syncthreads();
  float g1[kG1Reg];
#pragma unroll
  for (int t = 0; t < kG1Reg; ++t) g1[t] = 0.f;
  const int nG1 = I1 * R;
  const bool g1_in_regs = nG1 <= kG1Reg * kPassThreads;
  double esq = 0.0, tsq = 0.0;
  const long long nbatch = (nf + kNB - 1) / kNB;
  for (long long bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
    const long long f0 = bt * kNB;
    const int nb = (int)((nf - f0) < kNB ? (nf - f0) : kNB);
    // load the fiber tile (coalesced along i1) and the Khatri-Rao rows
    for (int e = threadIdx.x; e < I1 * kNB; e += blockDim.x) {
      const int f = e / I1, i = e - f * I1;
      E[i * (kNB + 1) + f] = (f < nb) ? __ldg(a.T + (size_t)I1 * (f0 + f) + i) : 0.f;
    }
    for (int e = threadIdx.x; e < kNB * R; e += blockDim.x) {
      const int f = e / R, r = e - f * R;
      float p = 0.f;
      if (f < nb) {
        long long rem = f0 + f;
        p = 1.f;
#pragma unroll
        for (int l = 1; l < L; ++l) { const int il = (int)(rem % d[l]); rem /= d[l]; p *= Ws[off[l] + r * d[l] + il]; }
      }
      KR[f * R + r] = p;
    }
    __syncthreads();
    // residual
    for (int e = threadIdx.x; e < I1 * kNB; e += blockDim.x) {
      const int i = e % I1, f = e / I1;
      float t = 0.f;
      for (int r = 0; r < R; ++r) t = fmaf(Ws[r * I1 + i], KR[f * R + r], t);
      const float x = E[i * (kNB + 1) + f];
      const float ev = (f < nb) ? x - t : 0.f;
      E[i * (kNB + 1) + f] = ev;
      esq += (double)ev * (double)ev;
      tsq += (double)x * (double)x;
    }
    __syncthreads();
    // G1 += E KR ; Q = E^T W1
    if (g1_in_regs) {
#pragma unroll
      for (int t = 0; t < kG1Reg; ++t) {
        const int o = threadIdx.x + t * kPassThreads;
        if (o < nG1) {
          const int r = o / I1, i = o - r * I1;
          float acc = g1[t];
          const float* er = E + i * (kNB + 1);
          for (int f = 0; f < kNB; ++f) acc = fmaf(er[f], KR[f * R + r], acc);
          g1[t] = acc;
        }
      }
    } else {
      for (int o = threadIdx.x; o < nG1; o += blockDim.x) {
        const int r = o / I1, i = o - r * I1;
        float acc = 0.f;
        for (int f = 0; f < kNB; ++f) acc = fmaf(E[i * (kNB + 1) + f], KR[f * R + r], acc);
        atomicAdd(a.G + o, acc);
      }
    }
    for (int o = threadIdx.x; o < kNB * R; o += blockDim.x) {
      const int r = o / kNB, f = o - r * kNB;
      float acc = 0.f;
      for (int i = 0; i < I1; ++i) acc = fmaf(E[i * (kNB + 1) + f], Ws[r * I1 + i], acc);
      Qs[f * R + r] = acc;
    }
    __syncthreads();
    // scatter q into the other modes
    for (int o = threadIdx.x; o < nb * R; o += blockDim.x) {
      const int f = o / R, r = o - f * R;
      int idx[kMaxL];
      long long rem = f0 + f;
#pragma unroll
      for (int l = 1; l < L; ++l) { idx[l] = (int)(rem % d[l]); rem /= d[l]; }
      const float q = Qs[f * R + r];
#pragma unroll
      for (int l = 1; l < L; ++l) {
        float p = q;
#pragma unroll
        for (int j = 1; j < L; ++j)
          if (j != l) p *= Ws[off[j] + r * d[j] + idx[j]];
        atomicAdd(Gs + off[l] + r * d[l] + idx[l], p);
      }
    }
    __syncthreads();
  }
  if (g1_in_regs) {
#pragma unroll
    for (int t = 0; t < kG1Reg; ++t) {
      const int o = threadIdx.x + t * kPassThreads;
      if (o < nG1 && g1[t] != 0.f) atomicAdd(a.G + o, g1[t]);
    }
  }
  for (int j = off[1] + threadIdx.x; j < n; j += blockDim.x)
    if (Gs[j] != 0.f) atomicAdd(a.G + j, Gs[j]);
  double v[2] = {esq, tsq};
  __shared__ double red[64];
  block_sum<2>(v, red);
  if (threadIdx.x == 0) {
    atomicAdd(a.esq, v[0]);
    if (a.want_tsq) atomicAdd(a.esq + 1, v[1]);
  }
}

static size_t pass_smem(int L, const long long* dims, int R) {
  size_t n = 0;
  for (int l = 0; l < L; ++l) n += (size_t)dims[l] * R;
  return (2 * n + (size_t)dims[0] * (kNB + 1) + 2 * (size_t)kNB * R) * sizeof(float);
}

__global__ void k_zero_pass(float* G, int n, double* esq, int want_tsq, const int* done) {
  if (done && *done) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) G[j] = 0.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) { esq[0] = 0.0; if (want_tsq) esq[1] = 0.0; }
}

cudaError_t launch_refine_pass(const RefinePassArgs& a, cudaStream_t st) {
  int n = 0;
  for (int l = 0; l < a.L; ++l) n += (int)a.dims[l] * a.R;
  k_zero_pass<<<16, 256, 0, st>>>(a.G, n, a.esq, a.want_tsq, a.done);
  count_launch();
  const size_t smem = pass_smem(a.L, a.dims, a.R);
  const void* fn = (a.L == 3) ? (const void*)k_refine_pass<3> : (const void*)k_refine_pass<4>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  long long nf = 1;
  for (int l = 1; l < a.L; ++l) nf *= a.dims[l];
  long long nbatch = (nf + kNB - 1) / kNB;
  long long blocks = nbatch < 2 * 152 ? nbatch : 2 * 152;
  if (blocks < 1) blocks = 1;
  if (a.L == 3) k_refine_pass<3><<<(unsigned)blocks, kPassThreads, smem, st>>>(a);
  else k_refine_pass<4><<<(unsigned)blocks, kPassThreads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

// ---- the single-CTA step ----------------------------------------------------------
size_t refine_step_smem_bytes(int L, const long long* dims, int R, int vec_in_smem) {
  size_t n = 0;
  for (int l = 0; l < L; ++l) n += (size_t)dims[l] * R;
  const size_t RR = (size_t)R * R;
  auto up = [](size_t x) { return (x + 3) & ~(size_t)3; };
  size_t f = up(L * RR) + up((size_t)L * L * RR) + 2 * up(L * RR) + 3 * up((size_t)L * R);
  if (vec_in_smem) f += 7 * up(n);
  return 128 * sizeof(double) + f * sizeof(float);
}

template <int L>
__global__ void __launch_bounds__(1024) k_refine_step(RefineStepArgs a) {
  if (*a.done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_stop;
  int dims[kMaxL];
  for (int l = 0; l < kMaxL; ++l) dims[l] = (l < L) ? (int)a.dims[l] : 1;
  Shape s; make_shape(s, L, dims, a.R);
  const int R = s.R;
  const size_t RR = (size_t)R * R;
  auto up = [](size_t x) { return (x + 3) & ~(size_t)3; };
  Bufs b{};
  b.red = reinterpret_cast<double*>(smem_raw);
  float* p = reinterpret_cast<float*>(smem_raw + 128 * sizeof(double));
  b.gram = p; p += up(L * RR);
  b.Pi2 = p; p += up((size_t)L * L * RR);
  b.Xm = p; p += up(L * RR);
  b.Ym = p; p += up(L * RR);
  b.msq = p; p += up((size_t)L * R);
  b.gam = p; p += up((size_t)L * R);
  b.sc = p; p += up((size_t)L * R);
  float* vb = a.vec_in_smem ? p : a.vecs;
  float** vecs[7] = {&b.W, &b.G, &b.X, &b.Rr, &b.P, &b.Z, &b.Tmp};
  for (int v = 0; v < 7; ++v) { *vecs[v] = vb; vb += up((size_t)s.n); }
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) { b.W[j] = a.W[j]; b.G[j] = a.G[j]; }
  double gm = 0.0;
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) gm = fmax(gm, (double)fabsf(a.G[j]));
  const double ginf = block_max(gm, b.red);   // also a barrier
  RefineState* st = a.state;
  if (threadIdx.x == 0) {
    s_stop = 0;
    const double esq = a.esq[0];
    if (a.j == 0) {
      st->normT = sqrt(a.esq[1]);
      st->F = 0.5 * esq;
      st->rel_err = st->normT > 0.0 ? sqrt(esq) / st->normT : 0.0;
      a.hist[0] = st->rel_err;
      if (!isfinite(esq)) { st->status = CPD_ERR_NUMERIC; s_stop = 1; }
    } else {
      double mu = st->mu;
      const double Fn = 0.5 * esq;
      const double gain = gain_update(st->F, Fn, st->pred_drop, mu);
      const double e = st->normT > 0.0 ? sqrt(esq) / st->normT : 0.0;
      st->mu = mu; st->F = Fn; st->rel_err = e; st->iters = a.j;
      a.hist[a.j] = e;
      write_trace(a.trace, a.trace_cap, a.trace_slot0 + a.j - 1, st->kglob, e, mu, gain,
                  -1, st->step, ginf, 1);
      int stop;
      if (!isfinite(esq) || !isfinite(st->step)) { st->status = CPD_ERR_NUMERIC; stop = CPD_STOP_NONE; s_stop = 1; }
      else {
        stop = stop_test(a.j, a.maxiter, a.tol, e, st->step, ginf, st->normT, a.hist);
        if (stop != CPD_STOP_NONE) { st->stop = stop; s_stop = 1; }
      }
    }
    if (s_stop) *a.done = 1;
  }
  __syncthreads();
  if (s_stop) return;
  const double mu = st->mu;
  grams_pi<L>(s, b);
  regularize<L>(s, b, mu);
  const int kglob = st->kglob + 1;
  const int maxit = cg_maxiter(kglob, a.seed, a.cg_a, a.cg_b);
  const int its = pcg<L>(s, b, mu, maxit, a.tol);
  double pred_drop, step;
  finish_step<L>(s, b, pred_drop, step);
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) a.W[j] = b.W[j];
  if (threadIdx.x == 0) {
    st->pred_drop = pred_drop; st->step = step; st->kglob = kglob; st->cg_total += its;
    if (a.trace && a.trace_slot0 + a.j < a.trace_cap)
      a.trace[(size_t)(a.trace_slot0 + a.j) * CPD_TRACE_FIELDS + 4] = its;
  }
}

cudaError_t launch_refine_step(const RefineStepArgs& a, int threads, size_t smem, cudaStream_t st) {
  const void* fn = (a.L == 3) ? (const void*)k_refine_step<3> : (const void*)k_refine_step<4>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (a.L == 3) k_refine_step<3><<<1, threads, smem, st>>>(a);
  else k_refine_step<4><<<1, threads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_refine_init(RefineState* s, const DevResult* core, int* done) {
  s->mu = core->mu; s->F = 0.0; s->normT = 0.0; s->pred_drop = 0.0; s->step = 0.0;
  s->kglob = core->kglob; s->cg_total = 0; s->stop = 0; s->status = CPD_OK; s->iters = 0;
  s->rel_err = 0.0;
  *done = (core->status != CPD_OK) ? 1 : 0;
}

cudaError_t launch_refine_init(RefineState* state, const DevResult* core_res, int* done, cudaStream_t st) {
  k_refine_init<<<1, 1, 0, st>>>(state, core_res, done);
  count_launch();
  return cudaGetLastError();
}

cudaError_t read_refine_result(const RefineState* state, int* iters, int* stop, int* cg_total,
                               double* rel_err, double* mu, int* status, cudaStream_t st) {
  static thread_local RefineState h;
  cudaError_t e = cudaMemcpyAsync(&h, state, sizeof(RefineState), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  *iters = h.iters; *stop = h.stop; *cg_total = h.cg_total; *rel_err = h.rel_err; *mu = h.mu;
  *status = h.status;
  return cudaSuccess;
}

}  // namespace cpdk
