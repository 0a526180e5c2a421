// Damped Gauss-Newton (Sec. 4.1.3) on a large core by a thread-block cluster:
// every CTA of the cluster runs the whole iteration on its own copy of the
// factors and CG vectors (Grams and Pi, regulariser, PCG with Theorem "Hv",
// update, balance: the small O(R^2 sum R_l) work, identical in every CTA),
// while the residual and MTTKRP gradient pass over the core -- the O(R N)
// part that bounds a single CTA once the core no longer fits its shared
// memory -- is split: CTA c owns a contiguous slice of the core's mode-1
// fibres, kept in its shared memory, and computes the partial gradient of its
// slice; the partials are summed through distributed shared memory in the
// same order by every CTA, so every CTA holds the same gradient and the
// replicated iteration stays identical across the cluster.  The stop
// decision of CTA 0 (which keeps the error history) is read by all.
//
// Per slice (fibres f, entries (i1, f)):
//   kr_f = prod_{l>=2} W_l[i_l(f), :]             (Khatri-Rao rows)
//   e = s - W1 kr_f^T,  fsq += ||e||^2             (residual, Sec. 4.1.3)
//   G1 += E KR                                     (mode-1 gradient)
//   q_f = e_f^T W1,  G_l[i_l, :] += q_f * prod_{j>=2, j!=l} W_j[i_j, :]
// the mode-2 term per fibre, the slower modes once per run of fibres that
// share (i_3, ..., i_L).
#include "kernels.h"
#include "solver.cuh"
#include "dgn_cta.cuh"

namespace cpdk {
namespace {

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
// every thread of every CTA of the cluster; release / acquire of shared memory
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ float cl_ldf(uint32_t addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ double cl_ldd(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ int cl_ldi(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// Slice of the core's mode-1 fibres owned by CTA `rank` of `size`.
__host__ __device__ inline void fibre_slice(long long n0, int rank, int size, long long& fa, long long& fb) {
  fa = n0 * rank / size;
  fb = n0 * (rank + 1) / size;
}

// Shared memory of one CTA: the solver's small buffers and vectors (as in the
// single-CTA solver), the partial gradient, and the slice buffers (core
// entries and residual, Khatri-Rao rows and q rows of the slice).
__host__ __device__ inline size_t cluster_smem_bytes(int L, const int* d, int R, int csize, int blk) {
  Shape s; make_shape(s, L, d, R);
  auto up = [](size_t x) { return (x + 3) & ~(size_t)3; };
  const long long n0 = s.N / s.d[0];
  const size_t nfs = (size_t)((n0 + csize - 1) / csize);
  size_t f = small_buf_floats(L, R, blk);
  f += 8 * up((size_t)s.n);                              // 7 solver vectors + the partial gradient
  f += 2 * up(nfs * (size_t)s.d[0]) + 2 * up(nfs * (size_t)R);
  return 128 * sizeof(double) + f * sizeof(float);
}

struct ClusterBufs {
  float* Gp;    // partial gradient of this CTA's slice (n)
  float* Ssl;   // slice entries, fibre-major (nfs x I1)
  float* Es;    // slice residual
  float* KRs;   // Khatri-Rao rows of the slice (nfs x R)
  float* Qs;    // q rows of the slice (nfs x R)
};

__device__ inline void carve_cluster(const Shape& s, Bufs& b, ClusterBufs& c, unsigned char* smem, long long nfs,
                                     int blk) {
  const int L = s.L, R = s.R;
  auto up = [](size_t x) { return (x + 3) & ~(size_t)3; };
  b.red = reinterpret_cast<double*>(smem);
  float* p = carve_small(b, reinterpret_cast<float*>(smem + 128 * sizeof(double)), L, R, blk);
  float** vecs[7] = {&b.W, &b.G, &b.X, &b.Rr, &b.P, &b.Z, &b.Tmp};
  for (int v = 0; v < 7; ++v) { *vecs[v] = p; p += up((size_t)s.n); }
  c.Gp = p; p += up((size_t)s.n);
  c.Ssl = p; p += up((size_t)nfs * s.d[0]);
  c.Es = p; p += up((size_t)nfs * s.d[0]);
  c.KRs = p; p += up((size_t)nfs * R);
  c.Qs = p;
  b.F = nullptr; b.Kb = nullptr; b.Bb = nullptr;
}

// Indices (i_2, ..., i_L) of global fibre F of the core (F = i_2 + I_2 (i_3 + ...)),
// in 32-bit arithmetic (a core that fits the cluster has far fewer than 2^31 fibres).
template <int L>
__device__ __forceinline__ void core_fibre(const Shape& s, long long F, int (&il)[kMaxL]) {
  unsigned rem = (unsigned)F;
#pragma unroll
  for (int l = 1; l < L; ++l) {
    const unsigned d = (unsigned)s.d[l], q = rem / d;
    il[l] = (int)(rem - q * d);
    rem = q;
  }
}

// Residual and gradient of the cluster's core: this CTA's slice [fa, fb) of
// fibres gives fsq and the partial gradient; after a cluster barrier every
// CTA sums all partials in rank order into b.G (and fsq, in every thread),
// and ginf = ||G||_inf (in thread 0).  The caller must pass a cluster barrier
// before the next call (the partials are overwritten).
template <int L>
__device__ void core_pass_cluster(const Shape& s, const Bufs& b, const ClusterBufs& c, long long fa, long long fb,
                                  double& fsq, double& ginf, double* s_fsq) {
  const int R = s.R, d0 = s.d[0];
  const int nfs = (int)(fb - fa);
  const float* W0 = b.W;
  // (1) Khatri-Rao rows of the slice; zero the partial gradient of modes 2..L
  for (int q = threadIdx.x; q < nfs * R; q += blockDim.x) {
    const int f = q / R, r = q - f * R;
    int il[kMaxL];
    core_fibre<L>(s, fa + f, il);
    float p = 1.f;
#pragma unroll
    for (int l = 1; l < L; ++l) p *= b.W[s.off[l] + r * s.d[l] + il[l]];
    c.KRs[q] = p;
  }
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) c.Gp[j] = 0.f;
  __syncthreads();
  // (2) residual e = s - W1 kr_f^T, entry by entry; fsq
  float accf[1] = {0.f};
  for (int e = threadIdx.x; e < nfs * d0; e += blockDim.x) {
    const int f = e / d0, i = e - f * d0;
    const float* kr = c.KRs + (size_t)f * R;
    float t = 0.f;
    for (int r = 0; r < R; ++r) t = fmaf(W0[r * d0 + i], kr[r], t);
    const float ev = c.Ssl[e] - t;
    c.Es[e] = ev;
    accf[0] = fmaf(ev, ev, accf[0]);
  }
  float acc[1];
  block_sum_f<1>(accf, acc, b.red);            // contains the barriers that publish Es
  // (3) mode-1 gradient G1[i, r] = sum_f e[i, f] kr[f, r] (the fibres split in
  // `parts` ranges, one thread per (i, r, range), partial sums added) and q_f = e_f^T W1
  const int parts = (int)blockDim.x / (d0 * R) > 1 ? (int)blockDim.x / (d0 * R) : 1;
  for (int q = threadIdx.x; q < d0 * R * parts; q += blockDim.x) {
    const int pr = q / (d0 * R), rq = q - pr * d0 * R, r = rq / d0, i = rq - r * d0;
    const int f0 = (int)((long long)nfs * pr / parts), f1 = (int)((long long)nfs * (pr + 1) / parts);
    float g = 0.f;
    for (int f = f0; f < f1; ++f) g = fmaf(c.Es[(size_t)f * d0 + i], c.KRs[(size_t)f * R + r], g);
    atomicAdd(&c.Gp[r * d0 + i], g);
  }
  for (int q = threadIdx.x; q < nfs * R; q += blockDim.x) {
    const int f = q / R, r = q - f * R;
    const float* ef = c.Es + (size_t)f * d0;
    const float* w = W0 + (size_t)r * d0;
    float g = 0.f;
    for (int i = 0; i < d0; ++i) g = fmaf(ef[i], w[i], g);
    c.Qs[q] = g;
  }
  __syncthreads();
  // (4) modes 2..L: mode 2 per fibre; the slower modes per run of fibres with
  // the same (i_3, ..., i_L) (run K = F / I_2), summed first over its fibres
  for (int q = threadIdx.x; q < nfs * R; q += blockDim.x) {
    const int f = q / R, r = q - f * R;
    int il[kMaxL];
    core_fibre<L>(s, fa + f, il);
    float p = c.Qs[q];
#pragma unroll
    for (int l = 2; l < L; ++l) p *= b.W[s.off[l] + r * s.d[l] + il[l]];
    atomicAdd(&c.Gp[s.off[1] + r * s.d[1] + il[1]], p);
  }
  if (L >= 3) {
    const int d1 = s.d[1];
    const long long k0 = fa / d1, k1 = (fb - 1) / d1;
    const int nrun = nfs > 0 ? (int)(k1 - k0 + 1) : 0;
    for (int q = threadIdx.x; q < nrun * R; q += blockDim.x) {
      const int g = q / R, r = q - g * R;
      const long long K = k0 + g;
      const long long lo = K * d1 > fa ? K * d1 : fa, hi = (K + 1) * d1 < fb ? (K + 1) * d1 : fb;
      float sum = 0.f;
      for (long long F = lo; F < hi; ++F) {
        const int i2 = (int)(F - K * d1);
        sum = fmaf(c.Qs[(size_t)(F - fa) * R + r], b.W[s.off[1] + r * d1 + i2], sum);
      }
      if constexpr (L == 3) {
        atomicAdd(&c.Gp[s.off[2] + r * s.d[2] + (int)K], sum);
      } else {
        const int i3 = (int)(K % s.d[2]), i4 = (int)(K / s.d[2]);
        atomicAdd(&c.Gp[s.off[2] + r * s.d[2] + i3], sum * b.W[s.off[3] + r * s.d[3] + i4]);
        atomicAdd(&c.Gp[s.off[3] + r * s.d[3] + i4], sum * b.W[s.off[2] + r * s.d[2] + i3]);
      }
    }
  }
  if (threadIdx.x == 0) *s_fsq = (double)acc[0];
  // (5) the cluster's sum, in rank order, into every CTA
  cl_sync();
  const uint32_t cs = cl_size();
  float gm = 0.f;
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) {
    float g = 0.f;
    for (uint32_t rk = 0; rk < cs; ++rk) g += cl_ldf(cl_map(c.Gp + j, rk));
    b.G[j] = g;
    gm = fmaxf(gm, fabsf(g));
  }
  // fsq: the partials summed in rank order by thread 0 only (FP64), then
  // published to every thread by block_max's barriers
  __shared__ double s_total;
  if (threadIdx.x == 0) {
    double fs = 0.0;
    for (uint32_t rk = 0; rk < cs; ++rk) fs += cl_ldd(cl_map(s_fsq, rk));
    s_total = fs;
  }
  const float gmax = block_max(gm, b.red);     // also publishes b.G and s_total
  fsq = s_total;
  ginf = 0.0;
  if (threadIdx.x == 0) ginf = (double)gmax;
}

template <int L>
__global__ void __launch_bounds__(1024) k_dgn_cluster(DgnArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ State st;
  __shared__ int chosen[kMaxR];
  __shared__ Shape s;
  __shared__ double s_fsq;
  __shared__ int s_ctl[2];                       // rank 0's stop and status, read by every CTA
  __shared__ int s_maxit;
  const uint32_t rank = cl_rank(), csize = cl_size();
  if (threadIdx.x == 0) {
    int dims[kMaxL];
    for (int l = 0; l < kMaxL; ++l) dims[l] = (l < L) ? (a.dev_dims ? a.dev_dims[l] : a.dims[l]) : 1;
    make_shape(s, L, dims, a.R);
  }
  __syncthreads();
  const long long n0 = s.N / s.d[0];
  long long fa, fb;
  fibre_slice(n0, (int)rank, (int)csize, fa, fb);
  Bufs b;
  ClusterBufs c;
  carve_cluster(s, b, c, smem_raw, (n0 + csize - 1) / csize, a.precond);
  const float* S = static_cast<const float*>(a.S);
  b.S = S;                                       // the MLSVD-energy start scans the whole core
  // ||S|| and mean|S| over the whole core (every CTA, the same sums), the slice into shared memory
  {
    float vf[2] = {0.f, 0.f};
    for (int e = threadIdx.x; e < s.N; e += blockDim.x) {
      const float x = S[e];
      vf[0] = fmaf(x, x, vf[0]);
      vf[1] += fabsf(x);
    }
    const long long e0 = fa * s.d[0], e1 = fb * s.d[0];
    for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) c.Ssl[e - e0] = S[e];
    double v[2];
    block_sum<2>(vf, v, b.red);
    if (threadIdx.x == 0) { st.normS = sqrt(v[0]); st.mu = v[1] / (double)s.N; }
  }
  if (rank == 0) fill_cg_table(a.cgtab, a.cgtab_len, a.seed, a.cg_a, a.cg_b);
  __syncthreads();
  const double normS = st.normS, meanabs = st.mu;
  double fsq, ginf;
  init_factors<L>(s, b, a.init, a.W0, a.seed, chosen);
  balance<L>(s, b);
  core_pass_cluster<L>(s, b, c, fa, fb, fsq, ginf, &s_fsq);
  if (threadIdx.x == 0) {
    st.mu = a.mu0 >= 0.0 ? a.mu0 : a.tau * meanabs;
    st.F = 0.5 * fsq;
    st.normS = normS;
    st.rel_err = normS > 0.0 ? sqrt(fsq) / normS : 0.0;
    st.grad_inf = ginf;
    st.kglob = a.k0; st.cg_total = 0; st.stop = 0; st.iters = 0;
    st.status = isfinite(fsq) ? CPD_OK : CPD_ERR_NUMERIC;
    if (rank == 0) a.hist[0] = st.rel_err;
  }
  cl_sync();                                     // partials read; the history's start written
  const double div = divergence_threshold(normS, a.tol);
  const bool bad0 = !isfinite(fsq);
  for (int k = 1; k <= a.maxiter && !bad0; ++k) {
    const double mu = st.mu;
    // the table rank 0 filled is visible to the cluster after the prologue's barrier
    if (threadIdx.x == 0)
      s_maxit = (a.k0 + k <= a.cgtab_len) ? a.cgtab[a.k0 + k] : cg_maxiter(a.k0 + k, a.seed, a.cg_a, a.cg_b);
    grams_pi<L>(s, b);                           // its first barrier publishes s_maxit
    if (a.precond) regularize_block<L>(s, b, mu);
    else regularize<L>(s, b, mu);
    const int maxit = s_maxit;
    const int its = a.precond ? pcg_block<L>(s, b, mu, maxit, a.tol)
                    : (s.n <= (int)blockDim.x) ? pcg_owned<L>(s, b, mu, maxit, a.tol) : pcg<L>(s, b, mu, maxit, a.tol);
    double pred_drop, step;
    finish_step<L>(s, b, pred_drop, step);
    core_pass_cluster<L>(s, b, c, fa, fb, fsq, ginf, &s_fsq);
    if (threadIdx.x == 0) {
      step = quick_sqrt(step);
      double m = st.mu;
      const double Fn = 0.5 * fsq;
      const double gain = gain_update(st.F, Fn, pred_drop, m, a.mu_min);
      const double e = st.normS > 0.0 ? quick_div(quick_sqrt(fsq), st.normS) : 0.0;
      st.mu = m; st.F = Fn; st.rel_err = e; st.grad_inf = ginf;
      st.cg_total += its; st.iters = k; st.kglob = a.k0 + k;
      s_ctl[0] = CPD_STOP_NONE;
      s_ctl[1] = CPD_OK;
      if (rank == 0) {
        a.hist[k] = e;
        write_trace(a.trace, a.trace_cap, a.trace_slot0 + k - 1, a.k0 + k, e, m, gain, its, step, ginf, 0);
        if (!isfinite(fsq) || !isfinite(step)) s_ctl[1] = CPD_ERR_NUMERIC;
        else s_ctl[0] = stop_test(k, a.maxiter, a.tol, e, step, ginf, div, a.hist);
      }
    }
    cl_sync();                                   // partials read by all; rank 0's decision visible
    if (threadIdx.x == 0) {
      const uint32_t r0 = 0;
      st.stop = cl_ldi(cl_map(&s_ctl[0], r0));
      st.status = cl_ldi(cl_map(&s_ctl[1], r0));
    }
    __syncthreads();
    if (st.stop != CPD_STOP_NONE || st.status != CPD_OK) break;
  }
  if (rank == 0) {
    for (int j = threadIdx.x; j < s.n; j += blockDim.x) a.W_out[j] = b.W[j];
    if (threadIdx.x == 0) {
      DevResult* r = a.res;
      r->status = bad0 ? CPD_ERR_NUMERIC : st.status; r->iters = st.iters; r->stop = st.stop;
      r->cg_total = st.cg_total; r->kglob = st.kglob; r->rel_err = st.rel_err; r->mu = st.mu;
      r->grad_inf = st.grad_inf; r->pad0 = 0; r->normS = st.normS;
    }
  }
  cl_sync();                                     // no CTA leaves while another may read its shared memory
}

}  // namespace

size_t dgn_cluster_smem_bytes_host(int L, const int* d, int R, int csize, int blk) {
  return cluster_smem_bytes(L, d, R, csize, blk);
}

// Cluster of `csize` CTAs (up to 16, the non-portable maximum) of `threads`
// threads each; cudaErrorInvalidConfiguration when the device cannot place
// such a cluster with this shared memory.
cudaError_t launch_dgn_cluster(int L, const DgnArgs& a, int threads, int csize, size_t smem, cudaStream_t st) {
  const void* fn = (L == 3) ? (const void*)k_dgn_cluster<3> : (const void*)k_dgn_cluster<4>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (csize > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)csize, 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg);
  if (e != cudaSuccess) return e;
  if (nclusters < 1) return cudaErrorInvalidConfiguration;
  e = (L == 3) ? cudaLaunchKernelEx(&cfg, k_dgn_cluster<3>, a) : cudaLaunchKernelEx(&cfg, k_dgn_cluster<4>, a);
  if (e != cudaSuccess) return e;
  count_launch();
  return cudaGetLastError();
}

}  // namespace cpdk
