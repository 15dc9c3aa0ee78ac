// Step kernels for Q = 14 with FP64 and FP32 storage (see lbm_step_impl.cuh);
// the 2-byte storage types are in lbm_step_q14h.cu, so the two compile in
// parallel.
#include "lbm_step_impl.cuh"

namespace lbm {

cudaError_t launch_step_q14_half(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st);

cudaError_t launch_step_q14(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st) {
  switch (d.storage) {
    case LBM_STORAGE_F64: return launch_typed<14, double, double>(d, n, b, st);
    case LBM_STORAGE_F32: return launch_typed<14, float, float>(d, n, b, st);
    case LBM_STORAGE_F16:
    case LBM_STORAGE_BF16: return launch_step_q14_half(d, n, b, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
