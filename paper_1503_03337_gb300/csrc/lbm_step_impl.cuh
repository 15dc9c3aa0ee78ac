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

// Even steps with two x-adjacent cells per thread (see update_pair_even; nx
// even); blockDim.x threads cover 2*blockDim.x cells of a row.  The 36
// packed values of a pair need more registers than one cell's 18, hence
// the looser cap.
template <int Q, typename S, bool FORCE>
__global__ void __launch_bounds__(256, 3) k_step_pair(Domain<float> d) {
  pdl_release();
  pdl_acquire();
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x0 >= d.nx || y >= d.ny) return;
  update_pair_even<Q, S, FORCE>(d, static_cast<S*>(d.f), x0 + d.nx * (y + d.ny * z));
}

// Odd steps with the cells ordered by kind.  Threads 0 .. interior-1 take
// the cells whose neighbours are all fluid and unwrapped (1 <= x <= nx-2,
// likewise y and z) in linear order, so every warp there runs the interior
// offset tables; a warp may span two rows, whose cells stay a few elements
// apart.  The threads after them take the other cells (update_cell_at's
// boundary variants): first x = 0 and x = nx-1 of the interior rows, then
// every cell of the boundary rows (the z = 0 and z = nz-1 planes, then y = 0
// and y = ny-1 of the planes between).  Needs nx, ny, nz >= 3.
struct OddSplit {
  int ix, iy;     // nx - 2, ny - 2
  int interior;   // (nx-2)(ny-2)(nz-2)
  int other;      // N - interior
};

__device__ __forceinline__ void odd_split_other(int nx, int ny, int nz, int g, int& x, int& y,
                                                int& z) {
  const int iy = ny - 2, ends = iy * (nz - 2) * 2;
  if (g < ends) {
    const int r = g >> 1;
    x = (g & 1) ? nx - 1 : 0;
    y = 1 + r % iy;
    z = 1 + r / iy;
    return;
  }
  g -= ends;
  int r = g / nx;
  x = g - r * nx;
  if (r < 2 * ny) {
    y = r % ny;
    z = r < ny ? 0 : nz - 1;
    return;
  }
  r -= 2 * ny;
  z = 1 + (r >> 1);
  y = (r & 1) ? ny - 1 : 0;
}

template <int Q, typename S, typename R, bool FORCE, bool SR>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 2 : 4)
    k_step_odd_split(Domain<R> d, OddSplit p) {
  pdl_release();
  pdl_acquire();
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  S* f = static_cast<S*>(d.f);
  if (g < p.interior) {
    const int r = g / p.ix;
    const int x = 1 + (g - r * p.ix);
    const int y = 1 + r % p.iy, z = 1 + r / p.iy;
    update_with_links<Q, S, R, true, FORCE, SR>(d, f, x + d.nx * (y + d.ny * z),
                                                make_links_interior(d), d.F, &d.key);
  } else if (g - p.interior < p.other) {
    int x, y, z;
    odd_split_other(d.nx, d.ny, d.nz, g - p.interior, x, y, z);
    update_cell_at<Q, S, R, true, FORCE, SR>(d, f, d.F, &d.key, x, y, z, -1, -1);
  }
}

constexpr bool kOddSplit = true;  // odd steps of domains with nx, ny, nz >= 3

template <typename R>
void launch_one(void (*kernel)(Domain<R>), const Domain<R>& d, dim3 grid, dim3 block, bool pdl,
                cudaStream_t st) {
  launch_pdl(kernel, grid, block, pdl, st, d);
}

template <int Q, typename S, typename R, bool SR>
void launch_parity(const Domain<R>& d, bool odd, bool force, dim3 grid, dim3 block,
                          const BlockShape& b, cudaStream_t st) {
  // two cells per thread: even steps of FP32 / FP16 / BF16 storage with nx
  // even and rounding to nearest; every other step runs one cell per thread
  if constexpr (sizeof(S) <= 4 && !SR) {
    if (b.cpt == 2 && !odd && d.nx % 2 == 0) {
      grid.x = (d.nx / 2 + block.x - 1) / block.x;
      if (force) launch_one(k_step_pair<Q, S, true>, d, grid, block, b.pdl != 0, st);
      else launch_one(k_step_pair<Q, S, false>, d, grid, block, b.pdl != 0, st);
      return;
    }
  }
  if (odd && kOddSplit && d.nx >= 3 && d.ny >= 3 && d.nz >= 3) {
    OddSplit p;
    p.ix = d.nx - 2;
    p.iy = d.ny - 2;
    p.interior = p.ix * p.iy * (d.nz - 2);
    p.other = (int)d.N - p.interior;
    const dim3 g1((unsigned)((d.N + 255) / 256)), b1(256);
    if (force) launch_pdl(k_step_odd_split<Q, S, R, true, SR>, g1, b1, b.pdl != 0, st, d, p);
    else launch_pdl(k_step_odd_split<Q, S, R, false, SR>, g1, b1, b.pdl != 0, st, d, p);
  } else if (odd) {
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
