// Refinement pass kernels for order-4 tensors (one translation unit per
// order so the instantiations compile in parallel).
#include "refine_pass.cuh"

namespace cpdk {

cudaError_t launch_refine_pass4(const RefinePassArgs& a, size_t smem, int threads, long long nbatch,
                                 cudaStream_t st) {
  return launch_pass_l<4>(a, smem, threads, nbatch, st);
}

}  // namespace cpdk
