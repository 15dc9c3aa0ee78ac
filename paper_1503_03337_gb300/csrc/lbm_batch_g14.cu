// Grouped batch kernels for Q = 14 (see lbm_batch.cuh).
#include "lbm_batch.cuh"

namespace lbm {
namespace batchk {

template <typename S, bool FORCE>
static void go(const GroupLaunch& g) {
  if constexpr (Stochastic<S>::enabled) {
    if (g.sr) {
      if (g.odd) k_group<14, S, true, true, FORCE><<<g.grid, g.block, 0, g.stream>>>(g.ents, g.count, g.tiles, g.per, g.s);
      else k_group<14, S, false, true, FORCE><<<g.grid, g.block, 0, g.stream>>>(g.ents, g.count, g.tiles, g.per, g.s);
      return;
    }
  }
  if (g.odd) k_group<14, S, true, false, FORCE><<<g.grid, g.block, 0, g.stream>>>(g.ents, g.count, g.tiles, g.per, g.s);
  else k_group<14, S, false, false, FORCE><<<g.grid, g.block, 0, g.stream>>>(g.ents, g.count, g.tiles, g.per, g.s);
}

template <typename S>
static void go_force(const GroupLaunch& g) {
  if (g.force) go<S, true>(g);
  else go<S, false>(g);
}

cudaError_t launch_group_q14(const GroupLaunch& g) {
  if (g.storage == LBM_STORAGE_F32) go_force<float>(g);
  else if (g.storage == LBM_STORAGE_F16) go_force<__half>(g);
  else go_force<__nv_bfloat16>(g);
  return cudaGetLastError();
}

}  // namespace batchk
}  // namespace lbm
