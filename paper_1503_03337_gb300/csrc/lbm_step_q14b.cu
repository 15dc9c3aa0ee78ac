// Step kernels for Q = 14 with BF16 storage (see lbm_step_impl.cuh).
#include "lbm_step_impl.cuh"

namespace lbm {

cudaError_t launch_step_q14_bf16(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st) {
  return launch_typed<14, __nv_bfloat16, float>(d, n, b, st);
}

}  // namespace lbm
