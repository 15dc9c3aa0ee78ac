// Persistent batch kernel: one cooperative launch runs a whole chunk of steps
// of every domain, with the bounded grid barrier between steps.  Its own
// file because it holds every (Q, storage, parity) variant in one kernel.
#include "lbm_batch.cuh"

namespace lbm {
namespace batchk {
namespace {

// A domain without a body force runs the force-free update, as in the
// single-domain and grouped kernels (so every mode computes bit-identical
// results).
// Each variant is a separate (not inlined) function: inlining all 24 of
// them into one kernel makes its compilation take minutes.
template <int Q, typename S, bool ODD, bool FORCE>
__device__ __noinline__ void persist_tile(const Domain<float>& d, int tx, int ty, int tz) {
  batch_tile<Q, S, ODD, false, true, FORCE>(d, tx, ty, tz);
}

template <int Q, typename S>
__device__ __forceinline__ void batch_tile_persist(const Domain<float>& d, int tx, int ty, int tz,
                                                   bool odd, bool force) {
  if (force) {
    if (odd) persist_tile<Q, S, true, true>(d, tx, ty, tz);
    else persist_tile<Q, S, false, true>(d, tx, ty, tz);
  } else {
    if (odd) persist_tile<Q, S, true, false>(d, tx, ty, tz);
    else persist_tile<Q, S, false, false>(d, tx, ty, tz);
  }
}


// Steps `nsteps` (persistent mode, cooperative launch, loads through L2
// only) of every domain in `ents` (none of them stochastically rounded).  Each CTA updates a contiguous
// range of `per` tiles of the launch's tile list every step and re-reads a
// domain descriptor only when its range crosses into the next domain.
__global__ void __launch_bounds__(256, 2) k_batch(const BatchEntry* __restrict__ ents, int nent,
                                                  int64_t total_tiles, int nsteps, int per,
                                                  GridBarrier* bar, long long spin_limit) {
  __shared__ Domain<float> sd;
  __shared__ int s_meta[7];  // Q, storage, odd, sr, tiles_x, tiles_y, force
  __shared__ int64_t s_begin, s_end;
  const int tid = threadIdx.x + blockDim.x * threadIdx.y;
  const int nthr = blockDim.x * blockDim.y;
  const int64_t t0 = (int64_t)blockIdx.x * per;
  const int64_t t1 = min(t0 + per, total_tiles);
  for (int s = 0; s < nsteps; ++s) {
    int64_t end = -1;
    TileCursor cur{};
    for (int64_t t = t0; t < t1; ++t) {
      if (t >= end) {
        const BatchEntry& e = ents[find_entry(ents, nent, t)];
        __syncthreads();  // every thread is done with the previous sd
        const int nw = (int)(sizeof(Domain<float>) / sizeof(int));
        for (int w = tid; w < nw; w += nthr)
          reinterpret_cast<int*>(&sd)[w] = reinterpret_cast<const int*>(&e.d)[w];
        __syncthreads();
        // the force and hash key of this step overwrite words of the copy
        if (tid == 0) {
          const int64_t n = e.n + s;
          if (e.period > 0.0) {
            const double c = cos(2.0 * M_PI * (double)n / e.period);
            for (int k = 0; k < 3; ++k) sd.F[k] = float(e.force[k] * c);
          } else {
            for (int k = 0; k < 3; ++k) sd.F[k] = float(e.force[k]);
          }
          sd.key = step_key(n);
          s_meta[0] = e.Q;
          s_meta[1] = e.storage;
          s_meta[2] = (int)(n & 1);
          s_meta[3] = e.rounding == LBM_ROUND_STOCHASTIC;
          s_meta[4] = e.tiles_x;
          s_meta[5] = e.tiles_y;
          s_meta[6] = e.force[0] != 0.0 || e.force[1] != 0.0 || e.force[2] != 0.0;
          s_begin = e.tile_begin;
          s_end = e.tile_begin + (int64_t)e.tiles_x * e.tiles_y * e.d.nz;
        }
        __syncthreads();
        end = s_end;
        cur.start((int)(t - s_begin), s_meta[4], s_meta[5]);
      }
      const bool odd = s_meta[2] != 0, force = s_meta[6] != 0;
      if (s_meta[0] == 14) {
        if (s_meta[1] == LBM_STORAGE_F32) batch_tile_persist<14, float>(sd, cur.tx, cur.ty, cur.tz, odd, force);
        else if (s_meta[1] == LBM_STORAGE_F16) batch_tile_persist<14, __half>(sd, cur.tx, cur.ty, cur.tz, odd, force);
        else batch_tile_persist<14, __nv_bfloat16>(sd, cur.tx, cur.ty, cur.tz, odd, force);
      } else {
        if (s_meta[1] == LBM_STORAGE_F32) batch_tile_persist<18, float>(sd, cur.tx, cur.ty, cur.tz, odd, force);
        else if (s_meta[1] == LBM_STORAGE_F16) batch_tile_persist<18, __half>(sd, cur.tx, cur.ty, cur.tz, odd, force);
        else batch_tile_persist<18, __nv_bfloat16>(sd, cur.tx, cur.ty, cur.tz, odd, force);
      }
      cur.next();
    }
    if (s + 1 < nsteps && !grid_sync(bar, spin_limit)) return;
  }
}

}  // namespace

cudaError_t launch_persistent(const PersistentLaunch& p) {
  const BatchEntry* ents = p.ents;
  int nent = p.nent;
  int64_t total = p.total_tiles;
  int nsteps = p.nsteps;
  int per = p.per;
  GridBarrier* bar = p.bar;
  long long spin = p.spin_limit;
  void* args[] = {&ents, &nent, &total, &nsteps, &per, &bar, &spin};
  return cudaLaunchCooperativeKernel((const void*)k_batch, p.grid, p.block, args, 0, p.stream);
}

int persistent_blocks_per_sm(int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}

}  // namespace batchk
}  // namespace lbm
