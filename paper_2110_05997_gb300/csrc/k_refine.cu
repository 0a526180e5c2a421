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
// Mode-1 fibers (I1 contiguous floats) in batches of kNB.  Thread i owns row
// i1 = i of every fiber: with kr_r = prod_{l>=2} W_l[i_l, r] (shared, float4
// broadcast loads) it forms t~ = sum_r W1[i1, r] kr_r (W1 row in registers),
// e = t - t~, ||e||^2, and accumulates G1[i1, :] += e kr in registers for the
// whole kernel.  Then Q = E^T W1 per fiber (float4 broadcast of W1 rows) and
// G_l[i_l, r] += q_r prod_{j>=2, j!=l} W_j[i_j, r] for l >= 2 (shared atomics).
constexpr int kNB = 32;

template <int L, int RMAX, int SLOTS>
__global__ void __launch_bounds__(256) k_refine_pass(RefinePassArgs a) {
  if (a.done && *a.done) return;
  extern __shared__ __align__(16) float sm[];
  const int R = a.R, R4 = (R + 3) & ~3;
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
  // shared: Ws (n) | W1r (I1 x R4, row-major) | Gs (n) | E (I1 x (kNB+1)) | KR (kNB x R4) | Qs (kNB x R4)
  float* Ws = sm;
  float* W1r = Ws + ((n + 3) & ~3);
  float* Gs = W1r + (size_t)I1 * R4;
  float* E = Gs + ((n + 3) & ~3);
  float* KR = E + (((size_t)I1 * (kNB + 1) + 3) & ~(size_t)3);
  float* Qs = KR + kNB * R4;
  for (int j = threadIdx.x; j < n; j += blockDim.x) { Ws[j] = a.W[j]; Gs[j] = 0.f; }
  for (int j = threadIdx.x; j < I1 * R4; j += blockDim.x) {
    const int i = j / R4, r = j - i * R4;
    W1r[j] = (r < R) ? a.W[r * I1 + i] : 0.f;
  }
  __syncthreads();
  // thread owns rows i1 = threadIdx.x + s * blockDim.x, s < SLOTS
  float w[SLOTS][RMAX], g1[SLOTS][RMAX];
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) {
    const int i = threadIdx.x + sl * blockDim.x;
#pragma unroll
    for (int r = 0; r < RMAX; ++r) { w[sl][r] = (i < I1 && r < R) ? W1r[i * R4 + r] : 0.f; g1[sl][r] = 0.f; }
  }
  double esq = 0.0, tsq = 0.0;
  const long long nbatch = (nf + kNB - 1) / kNB;
  for (long long bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
    const long long f0 = bt * kNB;
    const int nb = (int)((nf - f0) < kNB ? (nf - f0) : kNB);
    for (int e = threadIdx.x; e < kNB * R4; e += blockDim.x) {
      const int f = e / R4, r = e - f * R4;
      float p = 0.f;
      if (f < nb && r < R) {
        long long rem = f0 + f;
        p = 1.f;
#pragma unroll
        for (int l = 1; l < L; ++l) { const int il = (int)(rem % d[l]); rem /= d[l]; p *= Ws[off[l] + r * d[l] + il]; }
      }
      KR[e] = p;
    }
    __syncthreads();
#pragma unroll
    for (int sl = 0; sl < SLOTS; ++sl) {
      const int i = threadIdx.x + sl * blockDim.x;
      if (i >= I1) continue;
      float esqf = 0.f, tsqf = 0.f;
      const float* tp = a.T + (size_t)I1 * f0 + i;
      for (int f = 0; f < nb; ++f) {
        const float x = __ldg(tp + (size_t)I1 * f);
        const float4* k4 = reinterpret_cast<const float4*>(KR + f * R4);
        float kr[RMAX];
#pragma unroll
        for (int q = 0; q < RMAX / 4; ++q) {
          if (4 * q < R) {
            const float4 v = k4[q];
            kr[4 * q] = v.x; kr[4 * q + 1] = v.y; kr[4 * q + 2] = v.z; kr[4 * q + 3] = v.w;
          } else {
            kr[4 * q] = kr[4 * q + 1] = kr[4 * q + 2] = kr[4 * q + 3] = 0.f;
          }
        }
        float t = 0.f;
#pragma unroll
        for (int r = 0; r < RMAX; ++r) t = fmaf(w[sl][r], kr[r], t);
        const float ev = x - t;
        esqf = fmaf(ev, ev, esqf);
        tsqf = fmaf(x, x, tsqf);
#pragma unroll
        for (int r = 0; r < RMAX; ++r) g1[sl][r] = fmaf(ev, kr[r], g1[sl][r]);
        E[i * (kNB + 1) + f] = ev;
      }
      for (int f = nb; f < kNB; ++f) E[i * (kNB + 1) + f] = 0.f;
      esq += (double)esqf;
      tsq += (double)tsqf;
    }
    __syncthreads();
    // Q = E^T W1: job = (fiber f, 4 ranks), lanes over f
    const int nj = kNB * (R4 / 4);
    for (int job = threadIdx.x; job < nj; job += blockDim.x) {
      const int f = job % kNB, rg = job / kNB;
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4* wr = reinterpret_cast<const float4*>(W1r) + rg;
      for (int ii = 0; ii < I1; ++ii) {
        const float e = E[ii * (kNB + 1) + f];
        const float4 wv = wr[ii * (R4 / 4)];
        acc.x = fmaf(e, wv.x, acc.x); acc.y = fmaf(e, wv.y, acc.y);
        acc.z = fmaf(e, wv.z, acc.z); acc.w = fmaf(e, wv.w, acc.w);
      }
      reinterpret_cast<float4*>(Qs + f * R4)[rg] = acc;
    }
    __syncthreads();
    // scatter q into the other modes
    for (int o = threadIdx.x; o < nb * R; o += blockDim.x) {
      const int f = o / R, r = o - f * R;
      int idx[kMaxL];
      long long rem = f0 + f;
#pragma unroll
      for (int l = 1; l < L; ++l) { idx[l] = (int)(rem % d[l]); rem /= d[l]; }
      const float q = Qs[f * R4 + r];
#pragma unroll
      for (int l = 1; l < L; ++l) {
        float p = q;
#pragma unroll
        for (int j = 1; j < L; ++j)
          if (j != l) p *= Ws[off[j] + r * d[j] + idx[j]];
        atomicAdd(Gs + off[l] + r * d[l] + idx[l], p);
      }
    }
    // no barrier: the next batch's first writes (KR) are not read here, and
    // Qs / E are rewritten only after two more barriers
  }
#pragma unroll
  for (int sl = 0; sl < SLOTS; ++sl) {
    const int i = threadIdx.x + sl * blockDim.x;
    if (i >= I1) continue;
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
      if (r < R && g1[sl][r] != 0.f) atomicAdd(a.G + r * I1 + i, g1[sl][r]);
  }
  __syncthreads();
  for (int j = off[1] + threadIdx.x; j < n; j += blockDim.x)
    if (Gs[j] != 0.f) atomicAdd(a.G + j, Gs[j]);
  // per-thread FP64 partials -> per-warp FP64 sums -> global FP64 atomics
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    esq += __shfl_xor_sync(0xffffffffu, esq, o);
    tsq += __shfl_xor_sync(0xffffffffu, tsq, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(a.esq, esq);
    if (a.want_tsq) atomicAdd(a.esq + 1, tsq);
  }
}

static size_t pass_smem(int L, const long long* dims, int R) {
  size_t n = 0;
  for (int l = 0; l < L; ++l) n += (size_t)dims[l] * R;
  const size_t R4 = (R + 3) & ~3;
  const size_t n4 = (n + 3) & ~(size_t)3;
  return (2 * n4 + (size_t)dims[0] * R4 + (((size_t)dims[0] * (kNB + 1) + 3) & ~(size_t)3) +
          2 * (size_t)kNB * R4) * sizeof(float);
}

__global__ void k_zero_pass(float* G, int n, double* esq, int want_tsq, const int* done) {
  if (done && *done) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) G[j] = 0.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) { esq[0] = 0.0; if (want_tsq) esq[1] = 0.0; }
}

template <int L, int RMAX, int SLOTS>
static cudaError_t launch_pass_t(const RefinePassArgs& a, size_t smem, int threads, long long blocks,
                                 cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_refine_pass<L, RMAX, SLOTS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_refine_pass<L, RMAX, SLOTS><<<(unsigned)blocks, threads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

// Supported shapes: I1 <= 256 * SLOTS with RMAX * SLOTS <= 64 (I1 <= 1024 for
// R <= 16, I1 <= 512 for R <= 32, I1 <= 256 for R <= 64).
bool refine_pass_supported(int I1, int R) {
  if (R <= 16) return I1 <= 1024;
  if (R <= 32) return I1 <= 512;
  return I1 <= 256;
}

template <int L>
static cudaError_t launch_pass_l(const RefinePassArgs& a, size_t smem, int threads, long long blocks,
                                 cudaStream_t st) {
  const int slots = (int)((a.dims[0] + 255) / 256);
  if (a.R <= 16) {
    if (slots <= 1) return launch_pass_t<L, 16, 1>(a, smem, threads, blocks, st);
    if (slots <= 2) return launch_pass_t<L, 16, 2>(a, smem, threads, blocks, st);
    return launch_pass_t<L, 16, 4>(a, smem, threads, blocks, st);
  }
  if (a.R <= 32) {
    if (slots <= 1) return launch_pass_t<L, 32, 1>(a, smem, threads, blocks, st);
    return launch_pass_t<L, 32, 2>(a, smem, threads, blocks, st);
  }
  return launch_pass_t<L, 64, 1>(a, smem, threads, blocks, st);
}

cudaError_t launch_refine_pass(const RefinePassArgs& a, cudaStream_t st) {
  int n = 0;
  for (int l = 0; l < a.L; ++l) n += (int)a.dims[l] * a.R;
  if (!refine_pass_supported((int)a.dims[0], a.R)) return cudaErrorInvalidValue;
  k_zero_pass<<<16, 256, 0, st>>>(a.G, n, a.esq, a.want_tsq, a.done);
  count_launch();
  const size_t smem = pass_smem(a.L, a.dims, a.R);
  long long nf = 1;
  for (int l = 1; l < a.L; ++l) nf *= a.dims[l];
  const long long nbatch = (nf + kNB - 1) / kNB;
  const int threads = a.dims[0] >= 256 ? 256 : (int)((a.dims[0] + 31) / 32 * 32);
  int per_sm = (int)((227 * 1024) / (smem + 1024));
  const int by_threads = 2048 / threads;
  if (per_sm > by_threads) per_sm = by_threads;
  if (per_sm < 1) per_sm = 1;
  long long blocks = nbatch < (long long)per_sm * 152 ? nbatch : (long long)per_sm * 152;
  if (blocks < 1) blocks = 1;
  return a.L == 3 ? launch_pass_l<3>(a, smem, threads, blocks, st) : launch_pass_l<4>(a, smem, threads, blocks, st);
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
  __shared__ Shape s;
  if (threadIdx.x == 0) {
    int dims[kMaxL];
    for (int l = 0; l < kMaxL; ++l) dims[l] = (l < L) ? (int)a.dims[l] : 1;
    make_shape(s, L, dims, a.R);
  }
  __syncthreads();
  const int R = a.R;
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
  float gm = 0.f;
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) gm = fmaxf(gm, fabsf(a.G[j]));
  const double ginf = (double)block_max(gm, b.red);   // also a barrier
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
      const double e = st->normT > 0.0 ? quick_div(quick_sqrt(esq), st->normT) : 0.0;
      st->mu = mu; st->F = Fn; st->rel_err = e; st->iters = a.j;
      a.hist[a.j] = e;
      write_trace(a.trace, a.trace_cap, a.trace_slot0 + a.j - 1, st->kglob, e, mu, gain,
                  -1, st->step, ginf, 1);
      int stop;
      if (!isfinite(esq) || !isfinite(st->step)) { st->status = CPD_ERR_NUMERIC; stop = CPD_STOP_NONE; s_stop = 1; }
      else {
        stop = stop_test(a.j, a.maxiter, a.tol, e, st->step, ginf,
                         divergence_threshold(st->normT, a.tol), a.hist);
        if (stop != CPD_STOP_NONE) { st->stop = stop; s_stop = 1; }
      }
    }
    if (s_stop) *a.done = 1;
  }
  __syncthreads();
  if (s_stop) return;
  const double mu = st->mu;
  __shared__ int s_maxit;
  const int kglob = st->kglob + 1;
  if (threadIdx.x == 0)
    s_maxit = (kglob <= a.cgtab_len) ? a.cgtab[kglob] : cg_maxiter(kglob, a.seed, a.cg_a, a.cg_b);
  grams_pi<L>(s, b);                           // its first barrier publishes s_maxit
  regularize<L>(s, b, mu);
  const int maxit = s_maxit;
  const int its = pcg<L>(s, b, mu, maxit, a.tol);
  double pred_drop, step;
  finish_step<L>(s, b, pred_drop, step);
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) a.W[j] = b.W[j];
  if (threadIdx.x == 0) {
    st->pred_drop = pred_drop; st->step = quick_sqrt(step); st->kglob = kglob; st->cg_total += its;
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
