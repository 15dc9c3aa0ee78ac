// Step kernels of the single-domain path and their typed launchers.  Each
// lbm_step_q*.cu file instantiates them for one Q, so the variants compile in
// parallel.
#pragma once

#include <cmath>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"
#include "lbm_launch.cuh"
#include "lbm_staged.cuh"

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

template <typename R>
void launch_one(void (*kernel)(Domain<R>), const Domain<R>& d, dim3 grid, dim3 block, bool pdl,
                cudaStream_t st) {
  launch_pdl(kernel, grid, block, pdl, st, d);
}

// Can the row-staged kernel run this domain?  Every bulk copy must start on
// a 16-byte boundary and span a multiple of 16 bytes.
inline bool stage_fits(const Domain<float>& d) {
  return d.nx % 8 == 0 && d.nx >= 16 && reinterpret_cast<uintptr_t>(d.f) % 16 == 0;
}

constexpr int kStageSegTarget = 128;  // cells per segment aimed at (64 threads)

// Units, segment length, ring depth and per-cell work of one step of the
// row-staged kernel (see lbm_staged.cuh).
inline StagePlan stage_plan(const Domain<float>& d, bool odd, int elem_bytes) {
  StagePlan p{};
  int64_t rows;
  if (!odd) {
    p.x0 = 0;
    p.xlen = d.nx;
    p.row_lo = 0;
    p.rows_y = d.ny;
    rows = (int64_t)d.ny * d.nz;
    p.general = 0;
  } else {
    const int iy = d.ny > 2 ? d.ny - 2 : 0, iz = d.nz > 2 ? d.nz - 2 : 0;
    p.x0 = 1;
    p.xlen = d.nx - 2;
    p.row_lo = 1;
    p.rows_y = iy > 0 ? iy : 1;
    rows = (int64_t)iy * iz;
    const int nzp = d.nz > 1 ? 2 : 1, nyp = d.ny > 1 ? 2 : 1;
    const int64_t boundary_rows = (int64_t)nzp * d.ny + (int64_t)(d.nz > 2 ? d.nz - 2 : 0) * nyp;
    p.general = rows * 2 + boundary_rows * d.nx;
  }
  // balanced segments on the 8-element grid: segment j spans
  // [j*seg, (j+1)*seg) of the row, clipped to the staged range
  p.nseg = (d.nx + kStageSegTarget - 1) / kStageSegTarget;
  p.seg = ((d.nx + p.nseg - 1) / p.nseg + 7) / 8 * 8;
  p.nseg = (d.nx + p.seg - 1) / p.seg;
  p.units = rows * p.nseg;
  // ring depth: about half the shared memory of an SM holds copies in
  // flight with either depth; the shallower ring fits more CTAs (warps)
  p.stages = elem_bytes == 4 ? 2 : 3;
  return p;
}

template <int Q, typename S, bool ODD, bool FORCE>
void launch_staged_kernel(const Domain<float>& d, const StagePlan& p, bool pdl, cudaStream_t st) {
  auto kernel = k_step_staged<Q, S, ODD, FORCE>;
  const int threads = ((p.seg / 2 + 31) / 32) * 32;
  const size_t smem = stage_smem_bytes<Q, S>(p.seg, p.stages);
  // resident CTAs per SM for the last shape asked (shapes rarely change)
  static int cached_threads = 0, cached_nb = 0, sms = 0;
  static size_t cached_smem = 0;
  if (threads != cached_threads || smem != cached_smem) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) !=
            cudaSuccess ||
        nb < 1)
      nb = 1;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    cached_threads = threads;
    cached_smem = smem;
    cached_nb = nb;
  }
  int64_t want = p.units;
  const int64_t general_ctas = (p.general + threads - 1) / threads;
  if (want < general_ctas) want = general_ctas;
  int64_t grid = (int64_t)cached_nb * sms;
  if (grid > want) grid = want;
  if (grid < 1) grid = 1;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, d, p);
}

template <int Q, typename S>
void launch_staged(const Domain<float>& d, bool odd, bool force, bool pdl, cudaStream_t st) {
  const StagePlan p = stage_plan(d, odd, (int)sizeof(S));
  if (odd) {
    if (force) launch_staged_kernel<Q, S, true, true>(d, p, pdl, st);
    else launch_staged_kernel<Q, S, true, false>(d, p, pdl, st);
  } else {
    if (force) launch_staged_kernel<Q, S, false, true>(d, p, pdl, st);
    else launch_staged_kernel<Q, S, false, false>(d, p, pdl, st);
  }
}

template <int Q, typename S, typename R, bool SR>
void launch_parity(const Domain<R>& d, bool odd, bool force, dim3 grid, dim3 block,
                          const BlockShape& b, cudaStream_t st) {
  // row-staged (cells_per_thread 3): FP32 / FP16 / BF16 storage, rounding to
  // nearest, nx a multiple of 8 and >= 16.  Two cells per thread: even steps
  // of FP32 / FP16 / BF16 storage with nx even and rounding to nearest.
  // Every other step runs one cell per thread.
  if constexpr (sizeof(S) <= 4 && !SR) {
    if (b.cpt == 3 && stage_fits(d)) {
      launch_staged<Q, S>(d, odd, force, b.pdl != 0, st);
      return;
    }
    if (b.cpt == 2 && !odd && d.nx % 2 == 0) {
      grid.x = (d.nx / 2 + block.x - 1) / block.x;
      if (force) launch_one(k_step_pair<Q, S, true>, d, grid, block, b.pdl != 0, st);
      else launch_one(k_step_pair<Q, S, false>, d, grid, block, b.pdl != 0, st);
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
