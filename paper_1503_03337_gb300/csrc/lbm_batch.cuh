// Device side of the batched stepping (lbm_batch.cu): the descriptor table
// entry, the bounded grid barrier, the per-tile update and the grouped
// kernels.  The grouped kernels are instantiated per Q in lbm_batch_g14.cu /
// lbm_batch_g18.cu so that their variants compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

template <typename R>
Domain<R> to_domain(const DomainDesc& d, const double F[3]);

namespace batchk {

struct BatchEntry {
  Domain<float> d;  // F and key are set per step on the device
  int Q, storage, rounding;
  int tiles_x, tiles_y;
  int64_t tile_begin;  // first tile of this domain in the launch
  int64_t n;           // step counter of this domain before the launch
  double force[3];
  double period;
};

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int timed_out;
  int extra;  // test hook: arrivals the barrier waits for beyond the grid
};

// Bounded grid-wide barrier for a cooperative launch.  Returns false (in
// every thread of the CTA) if the wait timed out anywhere.
__device__ inline bool grid_sync(GridBarrier* g, long long spin_limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    volatile unsigned int* vgen = &g->gen;
    volatile int* vflag = &g->timed_out;
    const unsigned int gen = *vgen;
    __threadfence();
    const unsigned int expected = gridDim.x + (unsigned int)g->extra;
    if (atomicAdd(&g->count, 1u) == expected - 1) {
      atomicExch(&g->count, 0u);
      __threadfence();
      atomicAdd(&g->gen, 1u);
    } else {
      long long k = 0;
      while (*vgen == gen) {
        if (*vflag || ++k > spin_limit) {
          atomicExch(&g->timed_out, 1);
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    ok = !*vflag;
  }
  __syncthreads();
  return ok != 0;
}

// Tile (tx, ty, z) of a domain: blockDim.x cells along x by blockDim.y rows.
template <int Q, typename S, bool ODD, bool SR, bool CG, bool FORCE = true>
__device__ __forceinline__ void batch_tile(const Domain<float>& d, int tx, int ty, int z) {
  const int x = tx * blockDim.x + threadIdx.x;
  const int y = ty * blockDim.y + threadIdx.y;
  if (x >= d.nx || y >= d.ny) return;
  const int x_lo = tx * blockDim.x + (threadIdx.x & ~31);
  update_cell<Q, S, float, ODD, FORCE, SR, CG>(d, static_cast<S*>(d.f), x, y, z, x_lo,
                                               x_lo + 31);
}

template <int Q, typename S, bool CG>
__device__ __forceinline__ void batch_tile_dispatch(const Domain<float>& d, int tx, int ty,
                                                    int tz, bool odd, bool sr) {
  if constexpr (Stochastic<S>::enabled) {
    if (sr) {
      if (odd) batch_tile<Q, S, true, true, CG>(d, tx, ty, tz);
      else batch_tile<Q, S, false, true, CG>(d, tx, ty, tz);
      return;
    }
  }
  if (odd) batch_tile<Q, S, true, false, CG>(d, tx, ty, tz);
  else batch_tile<Q, S, false, false, CG>(d, tx, ty, tz);
}

// Walks the tiles of one domain in order (x fastest) without divisions.
struct TileCursor {
  int tx, ty, tz, nx, ny;
  __device__ void start(int local, int tiles_x, int tiles_y) {
    nx = tiles_x;
    ny = tiles_y;
    tx = local % nx;
    const int r = local / nx;
    ty = r % ny;
    tz = r / ny;
  }
  __device__ void next() {
    if (++tx == nx) {
      tx = 0;
      if (++ty == ny) {
        ty = 0;
        ++tz;
      }
    }
  }
};

// Grouped mode: the domains of one launch share Q, storage, rounding and
// parity, so the kernel is the single-domain update specialised at compile
// time.  Each CTA updates a contiguous range of `per` tiles (the group's
// tiles numbered domain after domain) and re-reads a domain descriptor only
// when its range crosses into the next domain.  FORCE = false groups hold
// only domains without a body force.
template <int Q, typename S, bool ODD, bool SR, bool FORCE>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 2 : 4)
    k_group(const BatchEntry* __restrict__ ents, int nent, int64_t tiles, int per, int s) {
  __shared__ Domain<float> sd;
  __shared__ int s_tx, s_ty;
  __shared__ int64_t s_begin, s_end;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int64_t t0 = (int64_t)blockIdx.x * per;
  const int64_t t1 = min(t0 + per, tiles);
  int64_t end = -1;  // first tile past the domain held in sd
  TileCursor cur{};
  for (int64_t t = t0; t < t1; ++t) {
    if (t >= end) {
      int lo = 0, hi = nent - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ents[mid].tile_begin <= t) lo = mid;
        else hi = mid - 1;
      }
      const BatchEntry& e = ents[lo];
      __syncthreads();  // every thread is done with the previous sd
      const int nw = (int)(sizeof(Domain<float>) / sizeof(int));
      for (int w = tid; w < nw; w += blockDim.x * blockDim.y)
        reinterpret_cast<int*>(&sd)[w] = reinterpret_cast<const int*>(&e.d)[w];
      __syncthreads();
      if (tid == 0) {
        const int64_t n = e.n + s;
        if (e.period > 0.0) {
          const double c = cos(2.0 * M_PI * (double)n / e.period);
          for (int k = 0; k < 3; ++k) sd.F[k] = float(e.force[k] * c);
        } else {
          for (int k = 0; k < 3; ++k) sd.F[k] = float(e.force[k]);
        }
        sd.key = step_key(n);
        s_tx = e.tiles_x;
        s_ty = e.tiles_y;
        s_begin = e.tile_begin;
        s_end = e.tile_begin + (int64_t)e.tiles_x * e.tiles_y * e.d.nz;
      }
      __syncthreads();
      end = s_end;
      cur.start((int)(t - s_begin), s_tx, s_ty);
    }
    batch_tile<Q, S, ODD, SR, false, FORCE>(sd, cur.tx, cur.ty, cur.tz);
    cur.next();
  }
}

// Launch of one group's grouped kernel for one step (per-Q files).
struct GroupLaunch {
  int storage, sr, force, odd;
  dim3 grid, block;
  cudaStream_t stream;
  const BatchEntry* ents;
  int count;
  int64_t tiles;
  int per, s;
};
struct PersistentLaunch {
  const BatchEntry* ents;
  int nent;
  int64_t total_tiles;
  int nsteps, per;
  GridBarrier* bar;
  long long spin_limit;
  dim3 grid, block;
  cudaStream_t stream;
};
cudaError_t launch_persistent(const PersistentLaunch& p);
int persistent_blocks_per_sm(int threads);

cudaError_t launch_group_q14(const GroupLaunch& g);
cudaError_t launch_group_q18(const GroupLaunch& g);
int group_blocks_per_sm(int threads);

}  // namespace batchk
}  // namespace lbm
