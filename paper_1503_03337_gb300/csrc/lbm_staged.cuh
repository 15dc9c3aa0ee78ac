// Row-staged step for FP32 / FP16 / BF16 storage (FP32 arithmetic).
//
// A unit of work is one segment of up to kStageSeg cells of one x-row.  For
// every population array b the CTA copies, with one bulk copy, the part of
// row b that the segment's cells read (and later write) into shared memory,
// updates the cells there in place, two x-adjacent cells per thread in
// packed FP32x2, and copies the part back with one bulk store.  Two buffers
// alternate, so the next unit's loads are in flight while the current unit
// collides; one thread issues all copies, so the bytes in flight per SM do
// not depend on how many warps are resident.
//
// Even steps (no neighbour access) stage every row, x = 0..nx-1, and need no
// links.  Odd steps pull f_a(x) from slot abar of x - c_a and push f*_a to
// slot a of x + c_a: array b is read and written at x + c_b for the same
// cells, so the region staged for b is the segment shifted by c_b (the rows
// y + c_by, z + c_bz, and one element along x, covered by an aligned
// superset 8 elements wider).  Only interior rows are staged on odd steps,
// and in them x = 8..nx-9, so that no staged cell has a wall, wrap or mirror
// link; the other cells (boundary rows and the first and last 8 cells of
// interior rows) take the per-cell path of update_cell_at in the same
// launch.  The write region of an array with c_bx = +-1 starts or ends one
// element off the 16-byte grid: its aligned middle goes out in the bulk
// store and its 8 ragged end elements as plain stores.
//
// Cells only touch their own slots (the AA property), so the partition into
// staged and per-cell cells needs no ordering, and the superset loads may
// read slots owned by other cells (never used) while those are rewritten.
//
// Requirements (checked by stage_plan): nx a multiple of 8 and >= 24, every
// copy address and size a multiple of 16 bytes (nx % 8 == 0 and the
// population buffer 16-byte aligned make them so).
#pragma once

#include <cstring>

#include "lbm_bulk.cuh"
#include "lbm_kernels.cuh"
#include "lbm_launch.cuh"

namespace lbm {

constexpr int kStageSeg = 256;  // cells per segment at most (two per thread)
constexpr int kStagePad = 8;    // elements of margin on each side of a buffer row
constexpr uint64_t kStageWaitNs = 2000000000ull;  // bounded wait for a unit's loads

struct StagePlan {
  int seg;         // cells per segment (a multiple of 8, <= kStageSeg)
  int x0, xlen;    // staged x-range of a staged row: [x0, x0 + xlen)
  int nseg;        // segments per staged row
  int row_lo;      // 0 (even: every row) or 1 (odd: interior rows)
  int rows_y;      // staged rows per z-plane (ny or ny - 2)
  int64_t units;   // staged rows * nseg
  int64_t general; // cells of the per-cell path (odd steps)
  int* error;      // host-mapped flag, set when a unit's loads time out
};

// Elements per array in a stage buffer.
__host__ __device__ constexpr int stage_row_len(int seg) { return seg + 2 * kStagePad; }

template <int Q, typename S>
__host__ __device__ constexpr size_t stage_smem_bytes(int seg) {
  return 2 * (size_t)Q * stage_row_len(seg) * sizeof(S);
}

// Number of populations with c_x != 0 (their write regions have ragged ends).
template <int Q>
__host__ __device__ constexpr int num_x_movers() {
  int n = 0;
  for (int a = 0; a < Q; ++a) n += Lattice<Q>::c(a, 0) != 0;
  return n;
}

// The pair of values at element k of a staged row (MIS: k is odd, the pair
// straddles two aligned words).
template <typename S, bool MIS>
__device__ __forceinline__ pf2 stage_get(const S* row, int k) {
  if constexpr (sizeof(S) == 4) {
    if constexpr (MIS) return pf2(row[k], row[k + 1]);
    const float2 v = *reinterpret_cast<const float2*>(row + k);
    return pf2(v.x, v.y);
  } else {
    using W = typename Pair2<S>::type;
    if constexpr (MIS) {
      const uint32_t w0 = *reinterpret_cast<const uint32_t*>(row + k - 1);
      const uint32_t w1 = *reinterpret_cast<const uint32_t*>(row + k + 1);
      const uint32_t m = __byte_perm(w0, w1, 0x5432);  // high half of w0, low half of w1
      W w;
      memcpy(&w, &m, sizeof(w));
      return Pair2<S>::unpack(w);
    } else {
      return Pair2<S>::unpack(*reinterpret_cast<const W*>(row + k));
    }
  }
}

template <typename S, bool MIS>
__device__ __forceinline__ void stage_put(S* row, int k, pf2 v) {
  if constexpr (sizeof(S) == 4) {
    if constexpr (MIS) {
      row[k] = v.v.x;
      row[k + 1] = v.v.y;
    } else {
      *reinterpret_cast<float2*>(row + k) = v.v;
    }
  } else {
    using W = typename Pair2<S>::type;
    const W w = Pair2<S>::pack(v);
    if constexpr (MIS) {
      uint32_t bits;
      memcpy(&bits, &w, sizeof(bits));
      unsigned short* r16 = reinterpret_cast<unsigned short*>(row);
      r16[k] = (unsigned short)(bits & 0xffffu);
      r16[k + 1] = (unsigned short)(bits >> 16);
    } else {
      *reinterpret_cast<W*>(row + k) = w;
    }
  }
}

// (y, z) of staged row r.
__device__ __forceinline__ void stage_row(const StagePlan& p, int64_t r, int& y, int& z) {
  y = p.row_lo + (int)(r % p.rows_y);
  z = p.row_lo + (int)(r / p.rows_y);
}

// Thread 0: the loads of unit u into buf, announced on bar.
template <int Q, typename S, bool ODD>
__device__ __forceinline__ void stage_issue_loads(const Domain<float>& d, const StagePlan& p,
                                                  int64_t u, S* buf, uint64_t* bar) {
  const int L = stage_row_len(p.seg);
  int y, z;
  stage_row(p, u / p.nseg, y, z);
  const int xa = p.x0 + (int)(u % p.nseg) * p.seg;
  const int len = min(p.seg, p.x0 + p.xlen - xa);
  constexpr int wide = ODD ? num_x_movers<Q>() : 0;  // arrays loaded 8 elements wider
  mbar_arrive_expect_tx(bar, (uint32_t)((Q * len + wide * kStagePad) * sizeof(S)));
  const S* f = static_cast<const S*>(d.f);
  [&]<int... B>(std::integer_sequence<int, B...>) {
    (
        [&] {
          constexpr int cx = ODD ? Lattice<Q>::c(B, 0) : 0;
          constexpr int cy = ODD ? Lattice<Q>::c(B, 1) : 0;
          constexpr int cz = ODD ? Lattice<Q>::c(B, 2) : 0;
          const int64_t row = ((int64_t)(z + cz) * d.ny + (y + cy)) * d.nx;
          const int src_x = cx < 0 ? xa - kStagePad : xa;
          const int dst = cx < 0 ? 0 : kStagePad;
          const int n = len + (cx != 0 ? kStagePad : 0);
          bulk_load(buf + B * L + dst, f + (int64_t)B * d.N + row + src_x,
                    (uint32_t)(n * sizeof(S)), bar);
        }(),
        ...);
  }(std::make_integer_sequence<int, Q>{});
}

// Thread 0: the bulk stores of unit u from buf (odd steps: the aligned part
// of each write region).
template <int Q, typename S, bool ODD>
__device__ __forceinline__ void stage_issue_stores(const Domain<float>& d, const StagePlan& p,
                                                   int64_t u, const S* buf) {
  const int L = stage_row_len(p.seg);
  int y, z;
  stage_row(p, u / p.nseg, y, z);
  const int xa = p.x0 + (int)(u % p.nseg) * p.seg;
  const int len = min(p.seg, p.x0 + p.xlen - xa);
  S* f = static_cast<S*>(d.f);
  [&]<int... A>(std::integer_sequence<int, A...>) {
    (
        [&] {
          constexpr int cx = ODD ? Lattice<Q>::c(A, 0) : 0;
          constexpr int cy = ODD ? Lattice<Q>::c(A, 1) : 0;
          constexpr int cz = ODD ? Lattice<Q>::c(A, 2) : 0;
          const int64_t row = ((int64_t)(z + cz) * d.ny + (y + cy)) * d.nx;
          // aligned part: cx = 0 all of [xa, xa+len); +1 [xa+8, xa+len);
          // -1 [xa, xa+len-8)
          const int x_first = cx > 0 ? xa + kStagePad : xa;
          const int n = len - (cx != 0 ? kStagePad : 0);
          if (n > 0)
            bulk_store(f + (int64_t)A * d.N + row + x_first,
                       buf + A * L + (x_first - xa + kStagePad), (uint32_t)(n * sizeof(S)));
        }(),
        ...);
  }(std::make_integer_sequence<int, Q>{});
}

// All threads, odd steps: the ragged ends of the write regions of the
// populations with c_x != 0, 8 elements each: c_x = +1 owns
// [xa+1, xa+len+1), whose elements xa+1..xa+7 and xa+len are outside the
// bulk store; c_x = -1 owns [xa-1, xa+len-1): xa-1 and xa+len-8..xa+len-2.
template <int Q, typename S>
__device__ __forceinline__ void stage_edge_stores(const Domain<float>& d, const StagePlan& p,
                                                  int64_t u, const S* buf) {
  constexpr int M = num_x_movers<Q>();
  const int L = stage_row_len(p.seg);
  int y, z;
  stage_row(p, u / p.nseg, y, z);
  const int xa = p.x0 + (int)(u % p.nseg) * p.seg;
  const int len = min(p.seg, p.x0 + p.xlen - xa);
  S* f = static_cast<S*>(d.f);
  for (int e = threadIdx.x; e < M * kStagePad; e += blockDim.x) {
    const int rank = e / kStagePad, j = e % kStagePad;
    [&]<int... A>(std::integer_sequence<int, A...>) {
      int r = 0;  // rank of A among the populations with c_x != 0
      (
          [&] {
            constexpr int cx = Lattice<Q>::c(A, 0);
            if constexpr (cx != 0) {
              if (r == rank) {
                constexpr int cy = Lattice<Q>::c(A, 1), cz = Lattice<Q>::c(A, 2);
                const int x = cx > 0 ? (j < kStagePad - 1 ? xa + 1 + j : xa + len)
                                     : (j == 0 ? xa - 1 : xa + len - kStagePad - 1 + j);
                const int64_t row = ((int64_t)(z + cz) * d.ny + (y + cy)) * d.nx;
                f[(int64_t)A * d.N + row + x] = buf[A * L + (x - xa + kStagePad)];
              }
              ++r;
            }
          }(),
          ...);
    }(std::make_integer_sequence<int, Q>{});
  }
}

// One thread's pair of cells (t: pair index within the unit's segment),
// updated in place in the stage buffer.
template <int Q, typename S, bool ODD, bool FORCE>
__device__ __forceinline__ void stage_update_pair(const Domain<float>& d, S* buf, int L,
                                                  int t) {
  const int k = kStagePad + 2 * t;
  pf2 fv[Q];
  [&]<int... A>(std::integer_sequence<int, A...>) {
    // pull: f_a(x) from array abar at x - c_a (even steps: array a at x)
    ((fv[A] = ODD ? stage_get<S, (Lattice<Q>::c(A, 0) != 0)>(
                        buf + opposite<Q>(A) * L, k - Lattice<Q>::c(A, 0))
                  : stage_get<S, false>(buf + A * L, k)),
     ...);
  }(std::make_integer_sequence<int, Q>{});
  pf2 ux, uy, uz;
  collide<Q, FORCE>(fv, d.s, d.F[0], d.F[1], d.F[2], ux, uy, uz);
  [&]<int... A>(std::integer_sequence<int, A...>) {
    // push: f*_a to array a at x + c_a (even steps: array abar at x)
    (
        [&] {
          if constexpr (ODD)
            stage_put<S, (Lattice<Q>::c(A, 0) != 0)>(buf + A * L, k + Lattice<Q>::c(A, 0),
                                                       fv[A]);
          else
            stage_put<S, false>(buf + opposite<Q>(A) * L, k, fv[A]);
        }(),
        ...);
  }(std::make_integer_sequence<int, Q>{});
}

// Cell g of the per-cell path of an odd step: the first and last 8 cells of
// the interior rows, then every cell of the boundary rows (the z = 0 and
// z = nz-1 planes, then y = 0 and y = ny-1 of the planes between).
__device__ __forceinline__ void stage_general_cell(const Domain<float>& d, int64_t g, int& x,
                                                   int& y, int& z) {
  const int iy = max(d.ny - 2, 0), iz = max(d.nz - 2, 0);
  const int64_t ends = (int64_t)iy * iz * 2 * kStagePad;
  if (g < ends) {
    const int64_t r = g / (2 * kStagePad);
    const int j = (int)(g % (2 * kStagePad));
    x = j < kStagePad ? j : d.nx - 2 * kStagePad + j;
    y = 1 + (int)(r % iy);
    z = 1 + (int)(r / iy);
    return;
  }
  g -= ends;
  const int nzp = d.nz > 1 ? 2 : 1;
  const int64_t plane_rows = (int64_t)nzp * d.ny;
  int64_t r = g / d.nx;
  x = (int)(g % d.nx);
  if (r < plane_rows) {
    y = (int)(r % d.ny);
    z = r < d.ny ? 0 : d.nz - 1;
    return;
  }
  r -= plane_rows;
  const int nyp = d.ny > 1 ? 2 : 1;
  z = 1 + (int)(r / nyp);
  y = (r % nyp) == 0 ? 0 : d.ny - 1;
}

template <int Q, typename S, bool ODD, bool FORCE>
__global__ void __launch_bounds__(kStageSeg / 2, 4)
    k_step_staged(Domain<float> d, StagePlan p) {
  extern __shared__ __align__(128) unsigned char stage_smem[];
  __shared__ __align__(8) uint64_t bar[2];
  const int L = stage_row_len(p.seg);
  S* const buf0 = reinterpret_cast<S*>(stage_smem);
  S* const buf1 = buf0 + Q * L;
  const int tid = threadIdx.x;
  pdl_release();
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
  pdl_acquire();
  const int64_t stride = gridDim.x;
  if (tid == 0 && (int64_t)blockIdx.x < p.units)
    stage_issue_loads<Q, S, ODD>(d, p, blockIdx.x, buf0, &bar[0]);
  uint32_t phase = 0;  // bit b: parity of the next completion of bar[b]
  int it = 0;
  for (int64_t u = blockIdx.x; u < p.units; u += stride, ++it) {
    const int b = it & 1;
    S* const buf = b ? buf1 : buf0;
    const bool next = u + stride < p.units;
    if (tid == 0 && next) {
      bulk_wait_read_all();  // the other buffer's stores (previous unit) have read it
      stage_issue_loads<Q, S, ODD>(d, p, u + stride, b ? buf0 : buf1, &bar[b ^ 1]);
    }
    const bool ok = mbar_wait_bounded(&bar[b], (phase >> b) & 1u, kStageWaitNs);
    phase ^= 1u << b;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        *(volatile int*)p.error = 1;
        // let the loads already issued for the next unit land before exiting
        if (next) mbar_wait_bounded(&bar[b ^ 1], (phase >> (b ^ 1)) & 1u, kStageWaitNs);
      }
      break;
    }
    const int len = min(p.seg, p.x0 + p.xlen - (p.x0 + (int)(u % p.nseg) * p.seg));
    if (2 * tid < len) stage_update_pair<Q, S, ODD, FORCE>(d, buf, L, tid);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      stage_issue_stores<Q, S, ODD>(d, p, u, buf);
      bulk_commit();
    }
    if constexpr (ODD) stage_edge_stores<Q, S>(d, p, u, buf);
    __syncthreads();  // buf is reloaded two units on
  }
  if (tid == 0) bulk_wait_all();
  if constexpr (ODD) {
    S* f = static_cast<S*>(d.f);
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + tid; g < p.general; g += step) {
      int x, y, z;
      stage_general_cell(d, g, x, y, z);
      update_cell_at<Q, S, float, true, FORCE>(d, f, d.F, &d.key, x, y, z, -1, -1);
    }
  }
}

}  // namespace lbm
