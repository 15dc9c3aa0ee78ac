// Grouped batch kernels for Q = 18 (see lbm_batch.cuh); the solo kernels
// are in lbm_batch_s18.cu, so the two compile in parallel.
#include "lbm_batch.cuh"

namespace lbm {
namespace batchk {

cudaError_t launch_group_q18(const GroupLaunch& g) {
  return launch_by_storage<18, GroupLaunch, GroupOp>(g);
}

int group_blocks_per_sm(int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_group<18, float, true, false, true>,
                                                    threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}

}  // namespace batchk
}  // namespace lbm
