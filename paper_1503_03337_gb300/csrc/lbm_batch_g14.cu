// Grouped batch kernels for Q = 14 (see lbm_batch.cuh); the solo kernels
// are in lbm_batch_s14.cu, so the two compile in parallel.
#include "lbm_batch.cuh"

namespace lbm {
namespace batchk {

cudaError_t launch_group_q14(const GroupLaunch& g) {
  return launch_by_storage<14, GroupLaunch, GroupOp>(g);
}

}  // namespace batchk
}  // namespace lbm
