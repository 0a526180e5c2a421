// BF16 tensor-core (tcgen05) Gram of the first-mode unfolding.
#include "kernels.h"

namespace cpdk {

size_t gram_bf16_tc_scratch_bytes(long long I, long long C) { (void)I; (void)C; return 0; }

cudaError_t launch_gram_bf16_tc(const float* T, long long I, long long C, float* G, float* scratch,
                                size_t scratch_bytes, cudaStream_t st) {
  (void)T; (void)I; (void)C; (void)G; (void)scratch; (void)scratch_bytes; (void)st;
  return cudaErrorNotSupported;
}

}  // namespace cpdk
