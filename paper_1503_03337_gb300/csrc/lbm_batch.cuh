// Device side of the batched stepping (lbm_batch.cu): the descriptor table
// entry, the bounded grid barrier, the per-tile update and the grouped
// kernels.  The grouped and solo kernels are instantiated per Q in
// lbm_batch_g14.cu / _g18.cu and lbm_batch_s14.cu / _s18.cu so that their
// variants compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstddef>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"
#include "lbm_launch.cuh"

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

// Force and stochastic-rounding key of one domain at one step, written for
// every domain and step of a chunk by k_batch_prepare before the step
// kernels read them (the force's FP64 cosine is then evaluated once per
// domain and step, not once per CTA).
struct StepDyn {
  float F[3];
  uint32_t key;
};
static_assert(sizeof(StepDyn) == 16, "StepDyn is four words");
static_assert(offsetof(Domain<float>, key) == offsetof(Domain<float>, F) + 3 * sizeof(float),
              "F and key are adjacent in Domain, as in StepDyn");
static_assert(sizeof(Domain<float>) % sizeof(int) == 0, "Domain is copied word by word");

// Index of the entry holding tile t: the last k with ents[k].tile_begin <= t
// (ents[0].tile_begin = 0, strictly increasing).  A 32-way search by one
// warp: each round probes 32 evenly spaced entries with one load per lane,
// so 1024 entries take two dependent loads.  Called by whole warps; every
// lane returns the same index.
__device__ __forceinline__ int find_entry(const BatchEntry* __restrict__ ents, int nent,
                                          int64_t t) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = nent;  // the answer lies in [lo, hi)
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) >> 5;
    const int j = lo + lane * step;
    const bool ok = j < hi && ents[j].tile_begin <= t;
    const unsigned m = __ballot_sync(0xffffffffu, ok);  // bit 0 is always set
    lo += (31 - __clz((int)m)) * step;
    hi = min(hi, lo + step);
  }
  return lo;
}

// Copy of entry e's descriptor into shared memory by all threads of the
// CTA, with the step's force and key taken from v when USE_DYN.
template <bool USE_DYN>
__device__ __forceinline__ void load_domain(Domain<float>& sd, const BatchEntry& e,
                                            const StepDyn* v, int tid, int nthr) {
  constexpr int kWords = (int)(sizeof(Domain<float>) / sizeof(int));
  constexpr int kF = (int)(offsetof(Domain<float>, F) / sizeof(int));
  for (int w = tid; w < kWords; w += nthr) {
    int x;
    if (USE_DYN && w >= kF && w < kF + 4) x = reinterpret_cast<const int*>(v)[w - kF];
    else x = reinterpret_cast<const int*>(&e.d)[w];
    reinterpret_cast<int*>(&sd)[w] = x;
  }
}

// Grouped mode: the domains of one launch share Q, storage, rounding and
// parity, so the kernel is the single-domain update specialised at compile
// time.  Each CTA updates a contiguous range of `per` tiles (the group's
// tiles numbered domain after domain) and re-reads a domain descriptor only
// when its range crosses into the next domain.  FORCE = false groups hold
// only domains without a body force.  dyn[k] is entry k's force and key at
// this step.
template <int Q, typename S, bool ODD, bool SR, bool FORCE>
__global__ void __launch_bounds__(256, sizeof(S) == 8 ? 2 : 4)
    k_group(const BatchEntry* __restrict__ ents, const StepDyn* __restrict__ dyn, int nent,
            int tiles, int per) {
  pdl_release();
  pdl_acquire();
  __shared__ Domain<float> sd;
  __shared__ int s_tx, s_ty, s_begin, s_end;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  const int t0 = blockIdx.x * per;  // a group holds fewer than 2^31 tiles
  const int t1 = min(t0 + per, tiles);
  int end = -1;  // first tile past the domain held in sd
  TileCursor cur{};
  for (int t = t0; t < t1; ++t) {
    if (t >= end) {
      const int k = find_entry(ents, nent, t);
      const BatchEntry& e = ents[k];
      __syncthreads();  // every thread is done with the previous sd
      load_domain<FORCE || SR>(sd, e, dyn + k, tid, nthr);
      if (tid == 0) {
        s_tx = e.tiles_x;
        s_ty = e.tiles_y;
        s_begin = (int)e.tile_begin;
        s_end = (int)(e.tile_begin + (int64_t)e.tiles_x * e.tiles_y * e.d.nz);
      }
      __syncthreads();
      end = s_end;
      cur.start(t - s_begin, s_tx, s_ty);
    }
    batch_tile<Q, S, ODD, SR, false, FORCE>(sd, cur.tx, cur.ty, cur.tz);
    cur.next();
  }
}

// Solo mode: a domain large enough to fill the device by itself runs as
// its own launch of the single-domain update (descriptor in the kernel's
// parameter space, one cell per thread).  With DYN the step's force and key
// come from the table (a time-periodic force or stochastic rounding); the
// loaded values occupy registers for the whole update, so those variants
// get a looser register cap.  Without DYN the descriptor holds the constant
// force and the kernel is the single-domain step kernel.
template <int Q, typename S, bool ODD, bool SR, bool FORCE, bool DYN>
__global__ void __launch_bounds__(256, DYN ? 3 : 4)
    k_solo(Domain<float> d, const StepDyn* __restrict__ dyn) {
  pdl_release();
  pdl_acquire();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= d.nx || y >= d.ny) return;
  const int x_lo = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  if constexpr (DYN)
    update_cell_at<Q, S, float, ODD, FORCE, SR>(d, static_cast<S*>(d.f), dyn->F, &dyn->key, x,
                                                y, z, x_lo, x_lo + 31);
  else
    update_cell<Q, S, float, ODD, FORCE, SR>(d, static_cast<S*>(d.f), x, y, z, x_lo, x_lo + 31);
}

// Launch of one group's grouped kernel for one step (per-Q files).
struct GroupLaunch {
  int storage, sr, force, odd;
  dim3 grid, block;
  cudaStream_t stream;
  const BatchEntry* ents;
  const StepDyn* dyn;
  int count;
  int tiles;
  int per;
};
// Launch of one solo domain for one step (dyn: force and key from the
// table; else d.F holds the constant force).
struct SoloLaunch {
  int storage, sr, force, odd, dyn_force;
  dim3 grid, block;
  cudaStream_t stream;
  Domain<float> d;
  const StepDyn* dyn;
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
cudaError_t launch_solo_q14(const SoloLaunch& g);
cudaError_t launch_solo_q18(const SoloLaunch& g);
int group_blocks_per_sm(int threads);

// Typed dispatch of the grouped and solo launches; each per-Q file
// instantiates these for its Q.
template <int Q, typename S, bool FORCE>
void launch_group_typed(const GroupLaunch& g) {
  if constexpr (Stochastic<S>::enabled) {
    if (g.sr) {
      if (g.odd)
        launch_pdl(k_group<Q, S, true, true, FORCE>, g.grid, g.block, true, g.stream, g.ents, g.dyn, g.count, g.tiles, g.per);
      else
        launch_pdl(k_group<Q, S, false, true, FORCE>, g.grid, g.block, true, g.stream, g.ents, g.dyn, g.count, g.tiles, g.per);
      return;
    }
  }
  if (g.odd)
    launch_pdl(k_group<Q, S, true, false, FORCE>, g.grid, g.block, true, g.stream, g.ents, g.dyn, g.count, g.tiles, g.per);
  else
    launch_pdl(k_group<Q, S, false, false, FORCE>, g.grid, g.block, true, g.stream, g.ents, g.dyn, g.count, g.tiles, g.per);
}

template <int Q, typename S, bool FORCE>
void launch_solo_typed(const SoloLaunch& g) {
  if constexpr (Stochastic<S>::enabled) {
    if (g.sr) {
      if (g.odd) launch_pdl(k_solo<Q, S, true, true, FORCE, true>, g.grid, g.block, true, g.stream, g.d, g.dyn);
      else launch_pdl(k_solo<Q, S, false, true, FORCE, true>, g.grid, g.block, true, g.stream, g.d, g.dyn);
      return;
    }
  }
  if constexpr (FORCE) {
    if (g.dyn_force) {
      if (g.odd) launch_pdl(k_solo<Q, S, true, false, true, true>, g.grid, g.block, true, g.stream, g.d, g.dyn);
      else launch_pdl(k_solo<Q, S, false, false, true, true>, g.grid, g.block, true, g.stream, g.d, g.dyn);
      return;
    }
  }
  if (g.odd) launch_pdl(k_solo<Q, S, true, false, FORCE, false>, g.grid, g.block, true, g.stream, g.d, g.dyn);
  else launch_pdl(k_solo<Q, S, false, false, FORCE, false>, g.grid, g.block, true, g.stream, g.d, g.dyn);
}

template <int Q, typename L, template <int, typename, bool> class Op>
cudaError_t launch_by_storage(const L& g) {
  if (g.storage == LBM_STORAGE_F32) {
    if (g.force) Op<Q, float, true>::run(g);
    else Op<Q, float, false>::run(g);
  } else if (g.storage == LBM_STORAGE_F16) {
    if (g.force) Op<Q, __half, true>::run(g);
    else Op<Q, __half, false>::run(g);
  } else {
    if (g.force) Op<Q, __nv_bfloat16, true>::run(g);
    else Op<Q, __nv_bfloat16, false>::run(g);
  }
  return cudaGetLastError();
}

template <int Q, typename S, bool FORCE>
struct GroupOp {
  static void run(const GroupLaunch& g) { launch_group_typed<Q, S, FORCE>(g); }
};
template <int Q, typename S, bool FORCE>
struct SoloOp {
  static void run(const SoloLaunch& g) { launch_solo_typed<Q, S, FORCE>(g); }
};

}  // namespace batchk
}  // namespace lbm
