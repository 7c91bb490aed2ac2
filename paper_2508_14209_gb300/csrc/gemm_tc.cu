// gemm_tc.cu — placeholder for the tcgen05 tensor-core Gaussian stage.
#include "msk_internal.h"
namespace msk {
size_t tc_gemm_workspace(int64_t, int64_t, int64_t, int) { return 0; }
int launch_tc_gemm(uint64_t, int64_t, int64_t, int64_t, const float*, int64_t, int, double*,
                   int64_t, void*, size_t, cudaStream_t) {
  return MSK_ENOTSUP;
}
}  // namespace msk
