// Step kernels for Q = 26 with FP16 and BF16 storage (see lbm_step_impl.cuh).
#include "lbm_step_impl.cuh"

namespace lbm {

cudaError_t launch_step_q26_half(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st) {
  if (d.storage == LBM_STORAGE_F16) return launch_typed<26, __half, float>(d, n, b, st);
  return launch_typed<26, __nv_bfloat16, float>(d, n, b, st);
}

}  // namespace lbm
