// Step kernels of the single-domain path and their typed launchers.  Each
// lbm_step_q*.cu file instantiates them for one Q, so the variants compile in
// parallel.
#pragma once

#include <cmath>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"
#include "lbm_launch.cuh"

namespace lbm {

template <typename R>
Domain<R> to_domain(const DomainDesc& d, const double F[3]);

template <int Q, typename S, typename R, bool ODD, bool FORCE, bool SR>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 2 : 4) k_step(Domain<R> d) {
  pdl_release();
  pdl_acquire();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  // a 32-wide x-range containing x; it is the calling warp's range when
  // blockDim.x is a multiple of 32 (then the path choice is warp-uniform)
  const int x_lo = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  const int x_hi = x_lo + 31;
  update_cell<Q, S, R, ODD, FORCE, SR>(d, static_cast<S*>(d.f), x, y, z, x_lo, x_hi);
}

// Two cells per thread (see update_two); blockDim.x threads cover
// 2*blockDim.x cells of a row, each warp 64 consecutive cells.
template <int Q, typename S, bool ODD, bool FORCE, bool SR>
__global__ void __launch_bounds__(256, 3) k_step2(Domain<float> d) {
  pdl_release();
  pdl_acquire();
  const int lane = threadIdx.x & 31;
  const int x_lo = blockIdx.x * (2 * blockDim.x) + (threadIdx.x >> 5) * 64;
  const int xa = x_lo + lane;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (xa >= d.nx || y >= d.ny) return;
  update_two<Q, S, ODD, FORCE, SR>(d, static_cast<S*>(d.f), xa, y, z, x_lo);
}

template <typename R>
void launch_one(void (*kernel)(Domain<R>), const Domain<R>& d, dim3 grid, dim3 block, bool pdl,
                cudaStream_t st) {
  launch_pdl(kernel, grid, block, pdl, st, d);
}

template <int Q, typename S, typename R, bool SR>
void launch_parity(const Domain<R>& d, bool odd, bool force, dim3 grid, dim3 block,
                          const BlockShape& b, cudaStream_t st) {
  if constexpr (sizeof(S) <= 4) {
    if (b.cpt == 2) {
      grid.x = (d.nx + 2 * block.x - 1) / (2 * block.x);
      if (odd) {
        if (force) launch_one(k_step2<Q, S, true, true, SR>, d, grid, block, b.pdl != 0, st);
        else launch_one(k_step2<Q, S, true, false, SR>, d, grid, block, b.pdl != 0, st);
      } else {
        if (force) launch_one(k_step2<Q, S, false, true, SR>, d, grid, block, b.pdl != 0, st);
        else launch_one(k_step2<Q, S, false, false, SR>, d, grid, block, b.pdl != 0, st);
      }
      return;
    }
  }
  if (odd) {
    if (force) launch_one(k_step<Q, S, R, true, true, SR>, d, grid, block, b.pdl != 0, st);
    else launch_one(k_step<Q, S, R, true, false, SR>, d, grid, block, b.pdl != 0, st);
  } else {
    if (force) launch_one(k_step<Q, S, R, false, true, SR>, d, grid, block, b.pdl != 0, st);
    else launch_one(k_step<Q, S, R, false, false, SR>, d, grid, block, b.pdl != 0, st);
  }
}

template <int Q, typename S, typename R>
cudaError_t launch_typed(const DomainDesc& dd, int64_t n, BlockShape b,
                                cudaStream_t st) {
  double F[3];
  force_at(dd, n, F);
  const bool force = F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0 || dd.period > 0.0;
  Domain<R> d = to_domain<R>(dd, F);
  d.key = step_key(n);
  dim3 block(b.bx, b.by, 1);
  dim3 grid((dd.nx + b.bx - 1) / b.bx, (dd.ny + b.by - 1) / b.by, dd.nz);
  const bool odd = (n & 1) != 0;
  if constexpr (Stochastic<S>::enabled) {
    if (dd.rounding == LBM_ROUND_STOCHASTIC) {
      launch_parity<Q, S, R, true>(d, odd, force, grid, block, b, st);
      return cudaGetLastError();
    }
  }
  launch_parity<Q, S, R, false>(d, odd, force, grid, block, b, st);
  return cudaGetLastError();
}

}  // namespace lbm
