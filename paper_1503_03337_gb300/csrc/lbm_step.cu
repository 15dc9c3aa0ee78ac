// Single-domain fused step kernels and their dispatch.
#include <cmath>
#include <map>
#include <mutex>
#include <utility>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

template <typename R>
Domain<R> to_domain(const DomainDesc& d, const double F[3]) {
  Domain<R> o{};
  o.f = d.f;
  o.nx = d.nx;
  o.ny = d.ny;
  o.nz = d.nz;
  o.N = d.N;
  for (int k = 0; k < 3; ++k) o.per[k] = d.per[k];
  o.moving = d.moving;
  for (int face = 0; face < 6; ++face)
    for (int k = 0; k < 3; ++k) o.uw[face][k] = R(d.uw[face][k]);
  o.s.sc = R(d.s[0]);
  o.s.se = R(d.s[1]);
  o.s.sq = R(d.s[2]);
  o.s.snu = R(d.s[3]);
  o.s.spi = R(d.s[4]);
  o.s.st = R(d.s[5]);
  for (int k = 0; k < 3; ++k) o.F[k] = R(F[k]);
  o.key = 0;
  if (d.Q == 14) fill_offsets<14>(o);
  else fill_offsets<18>(o);
  return o;
}
template Domain<double> to_domain<double>(const DomainDesc&, const double*);
template Domain<float> to_domain<float>(const DomainDesc&, const double*);

void force_at(const DomainDesc& d, int64_t n, double F[3]) {
  const double c = d.period > 0.0 ? std::cos(2.0 * M_PI * (double)n / d.period) : 1.0;
  for (int k = 0; k < 3; ++k) F[k] = d.force[k] * c;
}

BlockShape default_block(int nx, int ny) {
  int bx = 32;
  while (bx < nx && bx < 128) bx *= 2;
  int by = 256 / bx;
  while (by > 1 && by / 2 >= ny) by /= 2;
  return {bx, by, 1, 0};
}

uint32_t step_key(int64_t n) {
  return mix32(0x5eedu ^ (uint32_t(n) * 0x632be5abu) ^ uint32_t(uint64_t(n) >> 32));
}

// Bulk L2 prefetch of the populations the CTA `dist` launch positions ahead
// will read (blocks start in linear block order, so that CTA runs about one
// wave later).  For every row of that CTA's tile and every direction a, the
// row segment holding f_a is prefetched: slot a of the same row on even
// steps, slot abar of the row at y - cy, z - cz (x widened by one cell each
// way) on odd steps.  Segments are widened to 16-byte boundaries and clipped
// to the population buffer, whose size is `bytes`.  A hint only: it changes
// no value.
__device__ __forceinline__ void prefetch_l2(const char* p, uint32_t n) {
  const size_t g = __cvta_generic_to_global(p);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g), "r"(n) : "memory");
}

template <int Q, typename S, bool ODD, typename R>
__device__ __forceinline__ void prefetch_ahead(const Domain<R>& d, int cells_x, int dist) {
  const int64_t nb = (int64_t)gridDim.x * gridDim.y * gridDim.z;
  const int64_t b = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z) +
                    dist;
  if (dist <= 0 || b >= nb) return;
  const int bx = (int)(b % gridDim.x);
  const int64_t r = b / gridDim.x;
  const int by = (int)(r % gridDim.y), bz = (int)(r / gridDim.y);
  const int x0 = bx * cells_x;
  const int x1 = min(x0 + cells_x, d.nx);
  const int rows = blockDim.y;
  const int t = threadIdx.x + blockDim.x * threadIdx.y;
  const int64_t total = d.N * Q * (int64_t)sizeof(S);
  const char* base = static_cast<const char*>(d.f);
  for (int k = t; k < rows * Q; k += blockDim.x * blockDim.y) {
    const int row = k / Q, a = k - row * Q;
    int y = by * rows + row, z = bz;
    if (y >= d.ny) continue;
    int pop = a, xs = x0, xe = x1;
    if constexpr (ODD) {
      y -= Lattice<Q>::c(a, 1);
      z -= Lattice<Q>::c(a, 2);
      if (y < 0 || y >= d.ny || z < 0 || z >= d.nz) continue;
      pop = opposite<Q>(a);
      xs = max(x0 - 1, 0);
      xe = min(x1 + 1, d.nx);
    }
    int64_t lo = ((int64_t)pop * d.N + xs + (int64_t)d.nx * (y + (int64_t)d.ny * z)) *
                 (int64_t)sizeof(S);
    int64_t hi = lo + (int64_t)(xe - xs) * (int64_t)sizeof(S);
    lo &= ~int64_t(15);
    hi = (hi + 15) & ~int64_t(15);
    if (hi > total) hi = total & ~int64_t(15);
    if (hi > lo) prefetch_l2(base + lo, (uint32_t)(hi - lo));
  }
}

template <int Q, typename S, typename R, bool ODD, bool FORCE, bool SR>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 2 : 4) k_step(Domain<R> d) {
  prefetch_ahead<Q, S, ODD>(d, blockDim.x, d.prefetch);
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

// Two cells per thread (see update_pair); blockDim.x threads cover
// 2*blockDim.x cells of a row, each warp 64 consecutive cells.
template <int Q, typename S, bool ODD, bool FORCE, bool SR>
__global__ void __launch_bounds__(256, 2) k_step2(Domain<float> d) {
  const int lane = threadIdx.x & 31;
  const int x_lo = blockIdx.x * (2 * blockDim.x) + (threadIdx.x >> 5) * 64;
  const int xa = x_lo + lane;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  prefetch_ahead<Q, S, ODD>(d, 2 * blockDim.x, d.prefetch);
  if (xa >= d.nx || y >= d.ny) return;
  update_pair<Q, S, ODD, FORCE, SR>(d, static_cast<S*>(d.f), xa, y, z, x_lo);
}

// CTAs of `kernel` resident on the whole device at `threads` per CTA (one
// wave), cached per kernel and block size.
static int wave_ctas(const void* kernel, int threads) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_pair(kernel, threads);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 0;
  }
  const int w = per_sm * sms;
  cache[key] = w;
  return w;
}

template <typename K, typename R>
static void launch_one(K kernel, Domain<R> d, dim3 grid, dim3 block, int pf_waves,
                       cudaStream_t st) {
  d.prefetch = pf_waves > 0 ? pf_waves * wave_ctas((const void*)kernel, block.x * block.y) : 0;
  kernel<<<grid, block, 0, st>>>(d);
}

template <int Q, typename S, typename R, bool SR>
static void launch_parity(const Domain<R>& d, bool odd, bool force, dim3 grid, dim3 block,
                          const BlockShape& b, cudaStream_t st) {
  if constexpr (sizeof(S) <= 4) {
    if (b.cpt == 2) {
      grid.x = (d.nx + 2 * block.x - 1) / (2 * block.x);
      if (odd) {
        if (force) launch_one(k_step2<Q, S, true, true, SR>, d, grid, block, b.pf, st);
        else launch_one(k_step2<Q, S, true, false, SR>, d, grid, block, b.pf, st);
      } else {
        if (force) launch_one(k_step2<Q, S, false, true, SR>, d, grid, block, b.pf, st);
        else launch_one(k_step2<Q, S, false, false, SR>, d, grid, block, b.pf, st);
      }
      return;
    }
  }
  if (odd) {
    if (force) launch_one(k_step<Q, S, R, true, true, SR>, d, grid, block, b.pf, st);
    else launch_one(k_step<Q, S, R, true, false, SR>, d, grid, block, b.pf, st);
  } else {
    if (force) launch_one(k_step<Q, S, R, false, true, SR>, d, grid, block, b.pf, st);
    else launch_one(k_step<Q, S, R, false, false, SR>, d, grid, block, b.pf, st);
  }
}

template <int Q, typename S, typename R>
static cudaError_t launch_typed(const DomainDesc& dd, int64_t n, BlockShape b,
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

cudaError_t launch_step(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st) {
  if (d.N == 0) return cudaSuccess;
  if (d.Q == 14) {
    switch (d.storage) {
      case LBM_STORAGE_F64: return launch_typed<14, double, double>(d, n, b, st);
      case LBM_STORAGE_F32: return launch_typed<14, float, float>(d, n, b, st);
      case LBM_STORAGE_F16: return launch_typed<14, __half, float>(d, n, b, st);
      case LBM_STORAGE_BF16: return launch_typed<14, __nv_bfloat16, float>(d, n, b, st);
    }
  } else {
    switch (d.storage) {
      case LBM_STORAGE_F64: return launch_typed<18, double, double>(d, n, b, st);
      case LBM_STORAGE_F32: return launch_typed<18, float, float>(d, n, b, st);
      case LBM_STORAGE_F16: return launch_typed<18, __half, float>(d, n, b, st);
      case LBM_STORAGE_BF16: return launch_typed<18, __nv_bfloat16, float>(d, n, b, st);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
