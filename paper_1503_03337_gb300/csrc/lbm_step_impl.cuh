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

// Resident 256-thread blocks per SM the register budget is sized for: four
// (64 registers a thread) for Q = 14 and 18 with 4- or 2-byte storage, two
// for their FP64.  Q = 26 needs more: three for FP32 (80 registers, a few
// dozen bytes spilled, measured faster at 256^3 than two: 29.3 vs 28.2
// GLUPS), two for FP16 / BF16 (34.8 at three vs 36.2 at two), one for FP64.
// The wide kernels (64-bit offsets, Q*N >= 2^31) of Q = 14 and 18 take
// three blocks (80 registers): at four they spill 150-180 bytes.
template <int Q, typename S, bool WIDE = false>
constexpr int step_min_blocks() {
  if (Q == 26) return sizeof(S) == 8 ? 1 : (sizeof(S) == 4 ? 3 : 2);
  if (WIDE && sizeof(S) <= 4) return 3;
  return sizeof(S) == 8 ? 2 : 4;
}

// WIDE: 64-bit population offsets, for domains with Q*N >= 2^31.
template <int Q, typename S, typename R, bool ODD, bool FORCE, bool SR, bool WIDE = false>
__global__ void __launch_bounds__(256, step_min_blocks<Q, S, WIDE>()) k_step(Domain<R> d) {
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
  update_cell<Q, S, R, ODD, FORCE, SR, false, WIDE>(d, static_cast<S*>(d.f), x, y, z, x_lo,
                                                    x_hi);
}

// Even steps with two x-adjacent cells per thread (see update_pair_even; nx
// even); blockDim.x threads cover 2*blockDim.x cells of a row.  The 36
// packed values of a pair need more registers than one cell's 18: at three
// 256-thread blocks per SM (80 registers) a pair spills about 100 bytes a
// thread to local memory, and is still faster than at two blocks without
// spills (measured at 256^3: FP16 66.4 vs 62.7 GLUPS for Q18, 85.0 vs 81.7
// for Q14).
template <int Q, typename S, bool FORCE, bool SR>
__global__ void __launch_bounds__(256, 3) k_step_pair(Domain<float> d) {
  pdl_release();
  pdl_acquire();
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x0 >= d.nx || y >= d.ny) return;
  update_pair_even<Q, S, FORCE, SR>(d, static_cast<S*>(d.f), x0 + d.nx * (y + d.ny * z));
}

template <typename R>
void launch_one(void (*kernel)(Domain<R>), const Domain<R>& d, dim3 grid, dim3 block, bool pdl,
                cudaStream_t st) {
  launch_pdl(kernel, grid, block, pdl, st, d);
}

template <int Q, typename S, typename R, bool SR>
void launch_parity(const Domain<R>& d, bool odd, bool force, bool wide, dim3 grid, dim3 block,
                   const BlockShape& b, cudaStream_t st) {
  // Q*N >= 2^31: one cell per thread with 64-bit population offsets
  if (wide) {
    if (odd) {
      if (force) launch_one(k_step<Q, S, R, true, true, SR, true>, d, grid, block, b.pdl != 0, st);
      else launch_one(k_step<Q, S, R, true, false, SR, true>, d, grid, block, b.pdl != 0, st);
    } else {
      if (force) launch_one(k_step<Q, S, R, false, true, SR, true>, d, grid, block, b.pdl != 0, st);
      else launch_one(k_step<Q, S, R, false, false, SR, true>, d, grid, block, b.pdl != 0, st);
    }
    return;
  }
  // two cells per thread: even steps of FP32 / FP16 / BF16 storage with nx
  // even and no solid nodes, Q = 14 or 18 (the 52 packed values of a Q = 26
  // pair would not fit the registers); every other step runs one cell per
  // thread
  if constexpr (sizeof(S) <= 4 && Q != 26) {
    if (b.cpt == 2 && !odd && d.nx % 2 == 0 && !d.solid) {
      grid.x = (d.nx / 2 + block.x - 1) / block.x;
      if (force) launch_one(k_step_pair<Q, S, true, SR>, d, grid, block, b.pdl != 0, st);
      else launch_one(k_step_pair<Q, S, false, SR>, d, grid, block, b.pdl != 0, st);
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
  // the force-carrying update whenever the amplitude is nonzero (also at the
  // steps where a periodic force passes through zero), as the batch does
  const bool force = dd.force[0] != 0.0 || dd.force[1] != 0.0 || dd.force[2] != 0.0;
  Domain<R> d = to_domain<R>(dd, F);
  d.key = step_key(n);
  dim3 block(b.bx, b.by, 1);
  dim3 grid((dd.nx + b.bx - 1) / b.bx, (dd.ny + b.by - 1) / b.by, dd.nz);
  const bool odd = (n & 1) != 0;
  const bool wide = (int64_t)dd.Q * dd.N >= (int64_t(1) << 31);
  if constexpr (Stochastic<S>::enabled) {
    if (dd.rounding == LBM_ROUND_STOCHASTIC) {
      launch_parity<Q, S, R, true>(d, odd, force, wide, grid, block, b, st);
      return cudaGetLastError();
    }
  }
  launch_parity<Q, S, R, false>(d, odd, force, wide, grid, block, b, st);
  return cudaGetLastError();
}

}  // namespace lbm
