// Refinement pass kernels for order-3 tensors (one translation unit per
// order so the instantiations compile in parallel).
#include "refine_pass.cuh"

namespace cpdk {

cudaError_t launch_refine_pass3(const RefinePassArgs& a, size_t smem, int threads, long long nbatch,
                                 cudaStream_t st) {
  return launch_pass_l<3>(a, smem, threads, nbatch, st);
}

}  // namespace cpdk
