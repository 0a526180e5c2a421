// Single-CTA damped Gauss-Newton on a small tensor (the compressed core, or T
// itself when no compression is asked for): Sec. 4.1.3 of the thesis, all
// iterations in one launch, no host round trip.  Also the component kernels
// behind cpd_core_eval and cpd_jtj_apply, which run the same device code.
#include "kernels.h"
#include "solver.cuh"
#include "dgn_cta.cuh"

namespace cpdk {

template <int L>
__global__ void __launch_bounds__(1024) k_dgn_core(DgnArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dgn_run<L>(a, smem_raw);
}

// cpd_core_eval: one residual + gradient pass by the solver's own code.
template <int L>
__global__ void __launch_bounds__(1024) k_core_eval(CoreEvalArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Shape s;
  if (threadIdx.x == 0) make_shape(s, L, a.dims, a.R);
  __syncthreads();
  Bufs b; float* Sbuf;
  carve(s, b, smem_raw, a.gscratch, a.big_in_smem, &Sbuf);
  double nrm, meanabs;
  load_tensor(s, a.S, 0, Sbuf, b.red, nrm, meanabs);
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) b.W[j] = a.W[j];
  __syncthreads();
  double fsq, ginf;
  core_pass<L>(s, b, fsq, ginf);
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) a.g_out[j] = b.G[j];
  if (a.f_out)
    for (int e = threadIdx.x; e < s.N; e += blockDim.x) a.f_out[e] = b.F[e];
  if (threadIdx.x == 0) *a.fsq_out = fsq;
}

// cpd_jtj_apply: Grams, Pi matrices and Theorem "Hv" by the solver's own code.
template <int L>
__global__ void __launch_bounds__(1024) k_jtj_apply(JtjArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Shape s;
  if (threadIdx.x == 0) make_shape(s, L, a.dims, a.R);
  __syncthreads();
  Bufs b; float* Sbuf;
  carve(s, b, smem_raw, nullptr, 0, &Sbuf);   // no tensor-sized buffers used
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) { b.W[j] = a.W[j]; b.Tmp[j] = a.V[j]; }
  __syncthreads();
  grams_pi<L>(s, b);
  hv_xy<L>(s, b, b.Tmp);
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) {
    int l, i, r; decode_j<L>(s, j, l, i, r);
    a.out[j] = hv_entry<L>(s, b, b.Tmp, l, i, r);
  }
}

size_t dgn_smem_bytes_host(int L, const int* d, int R, int big_in_smem, int blk) {
  return dgn_smem_bytes(L, d, R, big_in_smem, blk);
}
size_t dgn_gscratch_floats_host(int L, const int* d, int R, int big_in_smem) {
  return dgn_gscratch_floats(L, d, R, big_in_smem);
}

cudaError_t launch_dgn_core(int L, const DgnArgs& a, int threads, size_t smem, cudaStream_t st) {
  const void* fn = (L == 3) ? (const void*)k_dgn_core<3> : (const void*)k_dgn_core<4>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (L == 3) k_dgn_core<3><<<1, threads, smem, st>>>(a);
  else k_dgn_core<4><<<1, threads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_core_eval(int L, const CoreEvalArgs& a, int threads, size_t smem, cudaStream_t st) {
  const void* fn = (L == 3) ? (const void*)k_core_eval<3> : (const void*)k_core_eval<4>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (L == 3) k_core_eval<3><<<1, threads, smem, st>>>(a);
  else k_core_eval<4><<<1, threads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_jtj_apply(int L, const JtjArgs& a, int threads, size_t smem, cudaStream_t st) {
  const void* fn = (L == 3) ? (const void*)k_jtj_apply<3> : (const void*)k_jtj_apply<4>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (L == 3) k_jtj_apply<3><<<1, threads, smem, st>>>(a);
  else k_jtj_apply<4><<<1, threads, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace cpdk
