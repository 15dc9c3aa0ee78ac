// Step kernels for Q = 26 (see lbm_step_impl.cuh).
#include "lbm_step_impl.cuh"

namespace lbm {

cudaError_t launch_step_q26(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st) {
  switch (d.storage) {
    case LBM_STORAGE_F64: return launch_typed<26, double, double>(d, n, b, st);
    case LBM_STORAGE_F32: return launch_typed<26, float, float>(d, n, b, st);
    case LBM_STORAGE_F16: return launch_typed<26, __half, float>(d, n, b, st);
    case LBM_STORAGE_BF16: return launch_typed<26, __nv_bfloat16, float>(d, n, b, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
