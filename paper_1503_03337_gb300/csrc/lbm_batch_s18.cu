// Solo batch kernels for Q = 18 (see lbm_batch.cuh).
#include "lbm_batch.cuh"

namespace lbm {
namespace batchk {

cudaError_t launch_solo_q18(const SoloLaunch& g) {
  return launch_by_storage<18, SoloLaunch, SoloOp>(g);
}

}  // namespace batchk
}  // namespace lbm
