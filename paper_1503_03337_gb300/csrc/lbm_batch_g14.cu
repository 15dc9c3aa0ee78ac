// Grouped and solo batch kernels for Q = 14 (see lbm_batch.cuh).
#include "lbm_batch.cuh"

namespace lbm {
namespace batchk {

cudaError_t launch_group_q14(const GroupLaunch& g) {
  return launch_by_storage<14, GroupLaunch, GroupOp>(g);
}

cudaError_t launch_solo_q14(const SoloLaunch& g) {
  return launch_by_storage<14, SoloLaunch, SoloOp>(g);
}

}  // namespace batchk
}  // namespace lbm
