// Step kernels for Q = 14 with FP16 storage (see lbm_step_impl.cuh); BF16 is
// in lbm_step_q14b.cu, so the two compile in parallel.
#include "lbm_step_impl.cuh"

namespace lbm {

cudaError_t launch_step_q14_bf16(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st);

cudaError_t launch_step_q14_half(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st) {
  if (d.storage == LBM_STORAGE_F16) return launch_typed<14, __half, float>(d, n, b, st);
  return launch_step_q14_bf16(d, n, b, st);
}

}  // namespace lbm
