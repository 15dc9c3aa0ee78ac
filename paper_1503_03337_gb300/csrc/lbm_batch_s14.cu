// Solo batch kernels for Q = 14 (see lbm_batch.cuh).
#include "lbm_batch.cuh"

namespace lbm {
namespace batchk {

cudaError_t launch_solo_q14(const SoloLaunch& g) {
  return launch_by_storage<14, SoloLaunch, SoloOp>(g);
}

}  // namespace batchk
}  // namespace lbm
