// Batched persistent solver for many small uneven CPDs.
#include "kernels.h"

extern "C" {

size_t cpd_batch_workspace_size(int B, const int* dims, const int* ranks, const cpd_options* opts) {
  (void)B; (void)dims; (void)ranks; (void)opts;
  return 0;
}

int cpd_batch_solve(int B, const float* T_packed, const int64_t* t_off, const int* dims,
                    const int* ranks, const cpd_options* opts, float* W_packed,
                    const int64_t* w_off, float* lam_packed, const int64_t* l_off,
                    cpd_info* infos, void* workspace, size_t ws_bytes, void* stream) {
  (void)B; (void)T_packed; (void)t_off; (void)dims; (void)ranks; (void)opts; (void)W_packed;
  (void)w_off; (void)lam_packed; (void)l_off; (void)infos; (void)workspace; (void)ws_bytes; (void)stream;
  return CPD_ERR_UNSUPPORTED;
}

}
