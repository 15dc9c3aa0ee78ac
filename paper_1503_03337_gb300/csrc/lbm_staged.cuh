// Row-staged step for FP32 / FP16 / BF16 storage (FP32 arithmetic).
//
// A unit of work is one segment of one x-row.  For every population array b
// the CTA's threads copy the part of row b that the segment's cells read
// (and later write) into shared memory in 16-byte chunks (cp.async, one
// chunk per thread and instruction, so a warp moves 512 bytes where the
// per-cell kernels move 64 or 128), update the cells there in place, two
// x-adjacent cells per thread in packed FP32x2, and write the part back in
// 16-byte chunks.  A ring of buffers keeps the copies of the next units in
// flight (commit groups) while the current unit collides.
//
// Even steps (no neighbour access) stage every row, x = 0..nx-1, and need no
// links.  Odd steps pull f_a(x) from slot abar of x - c_a and push f*_a to
// slot a of x + c_a: array b is read and written at x + c_b for the same
// cells, so the region staged for b is the segment shifted by c_b (the rows
// y + c_by, z + c_bz, and one element along x, covered by the aligned
// superset on the 8-element grid).  Only interior rows are staged on odd
// steps, and in them x = 1..nx-2, so that no staged cell has a wall, wrap or
// mirror link; the other cells (boundary rows and the ends x = 0, nx-1 of
// interior rows) take the per-cell path of update_cell_at in the same
// launch.  A write region that starts or ends off the 16-byte grid goes out
// as chunks of its aligned middle and plain stores of its ends.
//
// Cells only touch their own slots (the AA property), so the partition into
// staged and per-cell cells needs no ordering, and the superset loads may
// read slots owned by other cells (never used) while those are rewritten.
//
// Requirements (stage_fits): nx a multiple of 8 and >= 16 and the population
// buffer 16-byte aligned; then every chunk address is a multiple of 16 bytes.
#pragma once

#include <cstring>

#include "lbm_kernels.cuh"
#include "lbm_launch.cuh"

namespace lbm {

constexpr int kStageSeg = 256;      // cells per segment at most (two per thread)
constexpr int kStagePad = 8;        // elements of margin on each side of a buffer row
constexpr int kStageMaxStages = 4;  // buffers in the ring

struct StagePlan {
  int seg;         // cells per segment (a multiple of 8, <= kStageSeg); segment j
                   // of a row spans [j*seg, (j+1)*seg) clipped to the staged range
  int x0, xlen;    // staged x-range of a staged row: [x0, x0 + xlen)
  int nseg;        // segments per staged row
  int row_lo;      // 0 (even: every row) or 1 (odd: interior rows)
  int rows_y;      // staged rows per z-plane (ny or ny - 2)
  int stages;      // buffers in the ring (2..kStageMaxStages)
  int64_t units;   // staged rows * nseg (< 2^31)
  int64_t general; // cells of the per-cell path (odd steps)
};

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
// This thread's copies older than its newest N groups are complete.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Elements per array in a stage buffer.
__host__ __device__ constexpr int stage_row_len(int seg) { return seg + 2 * kStagePad; }

template <int Q, typename S>
__host__ __device__ constexpr size_t stage_smem_bytes(int seg, int stages) {
  return (size_t)stages * Q * stage_row_len(seg) * sizeof(S);
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


__host__ __device__ __forceinline__ int floor8(int v) { return v & ~7; }
__host__ __device__ __forceinline__ int ceil8(int v) { return (v + 7) & ~7; }

// Unit u: its row, the aligned base xb of its segment, and its staged cells
// [xa, xa + len).  Element x of a staged array row sits at buffer index
// x - xb + kStagePad.
struct StageUnit {
  int y, z, xb, xa, len;
};

__device__ __forceinline__ StageUnit stage_unit(const StagePlan& p, int u) {
  StageUnit s;
  const int r = u / p.nseg;
  s.y = p.row_lo + r % p.rows_y;
  s.z = p.row_lo + r / p.rows_y;
  s.xb = (u - r * p.nseg) * p.seg;
  s.xa = max(s.xb, p.x0);
  s.len = min(s.xb + p.seg, p.x0 + p.xlen) - s.xa;
  return s;
}

// Per-array shift of the staged regions, in shared memory for the whole
// kernel: the element offset of array b's staged row from the unit's row
// (b*N plus the y and z shifts on odd steps) and its x shift.
template <int Q>
struct StageShift {
  long long goff[Q];
  int cx[Q];
};

template <int Q, bool ODD>
__device__ __forceinline__ void stage_fill_shift(StageShift<Q>& t, const Domain<float>& d) {
  for (int b = threadIdx.x; b < Q; b += blockDim.x) {
    int cx = 0, cy = 0, cz = 0;
    if constexpr (ODD) {
      [&]<int... B>(std::integer_sequence<int, B...>) {
        ((b == B ? (cx = Lattice<Q>::c(B, 0), cy = Lattice<Q>::c(B, 1),
                    cz = Lattice<Q>::c(B, 2), 0)
                 : 0),
         ...);
      }(std::make_integer_sequence<int, Q>{});
    }
    t.goff[b] = (long long)b * d.N + ((long long)cz * d.ny + cy) * d.nx;
    t.cx[b] = cx;
  }
}

// All threads: the copies of unit t into buf.  Array b is staged over the
// aligned superset [floor8(xa + c), ceil8(xa + len + c)) of its region, c
// its x shift; chunk j of a buffer row holds elements xb - 8 + j*V .. + V-1
// (V = 16 / sizeof(S)).
template <int Q, typename S>
__device__ __forceinline__ void stage_issue_loads(const Domain<float>& d, const StagePlan& p,
                                                  const StageShift<Q>& sh, const StageUnit& t,
                                                  S* buf) {
  constexpr int V = 16 / sizeof(S);
  const int L = stage_row_len(p.seg), CH = L / V;
  const S* f = static_cast<const S*>(d.f) + ((long long)t.z * d.ny + t.y) * d.nx;
  for (int e = threadIdx.x; e < Q * CH; e += blockDim.x) {
    const int b = e / CH, j = e - b * CH;
    const int x = t.xb - kStagePad + j * V, c = sh.cx[b];
    if (x >= floor8(t.xa + c) && x < ceil8(t.xa + t.len + c))
      cp_async16(buf + b * L + j * V, f + sh.goff[b] + x);
  }
}

// All threads: the aligned middle [ceil8(xa + c), floor8(xa + len + c)) of
// each write region in 16-byte chunks, then (odd steps) its ragged ends,
// fewer than 8 elements on either side, as plain stores (slot j < 8 of an
// array: left end, j >= 8: right end).
template <int Q, typename S, bool ODD>
__device__ __forceinline__ void stage_stores(const Domain<float>& d, const StagePlan& p,
                                             const StageShift<Q>& sh, const StageUnit& t,
                                             const S* buf) {
  constexpr int V = 16 / sizeof(S);
  const int L = stage_row_len(p.seg), CH = L / V;
  S* f = static_cast<S*>(d.f) + ((long long)t.z * d.ny + t.y) * d.nx;
  for (int e = threadIdx.x; e < Q * CH; e += blockDim.x) {
    const int a = e / CH, j = e - a * CH;
    const int x = t.xb - kStagePad + j * V, c = sh.cx[a];
    if (x >= ceil8(t.xa + c) && x < floor8(t.xa + t.len + c))
      *reinterpret_cast<uint4*>(f + sh.goff[a] + x) =
          *reinterpret_cast<const uint4*>(buf + a * L + j * V);
  }
  if constexpr (ODD) {
    for (int e = threadIdx.x; e < Q * 2 * kStagePad; e += blockDim.x) {
      const int a = e / (2 * kStagePad), j = e % (2 * kStagePad);
      const int first = t.xa + sh.cx[a], end = t.xa + t.len + sh.cx[a];
      const int a0 = ceil8(first), a1 = floor8(end);
      const int x = j < kStagePad ? first + j : max(a0, a1) + (j - kStagePad);
      if (j < kStagePad ? x < min(a0, end) : x < end)
        f[sh.goff[a] + x] = buf[a * L + (x - t.xb + kStagePad)];
    }
  }
}

// One thread's pair of cells xb + 2t, xb + 2t + 1, updated in place in the
// stage buffer.  A pair may hold one cell outside the unit's staged range
// (the first or last cell of a row on odd steps): its values land only in
// slots no staged cell reads and no store of this unit writes.
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

// Cell g of the per-cell path of an odd step: x = 0 and x = nx-1 of the
// interior rows, then every cell of the boundary rows (the z = 0 and
// z = nz-1 planes, then y = 0 and y = ny-1 of the planes between).
__device__ __forceinline__ void stage_general_cell(const Domain<float>& d, int64_t g, int& x,
                                                   int& y, int& z) {
  const int iy = max(d.ny - 2, 0), iz = max(d.nz - 2, 0);
  const int64_t ends = (int64_t)iy * iz * 2;
  if (g < ends) {
    const int64_t r = g >> 1;
    x = (g & 1) ? d.nx - 1 : 0;
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
  __shared__ StageShift<Q> sh;
  const int L = stage_row_len(p.seg);
  const int K = p.stages;
  S* const base = reinterpret_cast<S*>(stage_smem);
  const int tid = threadIdx.x;
  pdl_release();
  stage_fill_shift<Q, ODD>(sh, d);
  __syncthreads();
  pdl_acquire();
  const int stride = gridDim.x, units = (int)p.units;
  // prologue: units 0..K-2 of this CTA into stages 0..K-2, one group each
  for (int s = 0; s < K - 1; ++s) {
    const int v = blockIdx.x + s * stride;
    if (v < units) stage_issue_loads<Q, S>(d, p, sh, stage_unit(p, v), base + s * Q * L);
    cp_async_commit();
  }
  int s = 0;  // stage of the current unit
  for (int u = blockIdx.x; u < units; u += stride) {
    S* const buf = base + s * Q * L;
    const int ahead = s == 0 ? K - 1 : s - 1;  // stage of unit u + (K-1)*stride
    const int v = u + (K - 1) * stride;
    if (v < units) stage_issue_loads<Q, S>(d, p, sh, stage_unit(p, v), base + ahead * Q * L);
    cp_async_commit();
    // all but the newest K-1 groups done: this unit's copies have landed
    if (K == 4) cp_async_wait<3>();
    else if (K == 3) cp_async_wait<2>();
    else cp_async_wait<1>();
    __syncthreads();
    const StageUnit t = stage_unit(p, u);
    if (t.xb + 2 * tid + 1 >= t.xa && t.xb + 2 * tid < t.xa + t.len)
      stage_update_pair<Q, S, ODD, FORCE>(d, buf, L, tid);
    __syncthreads();
    stage_stores<Q, S, ODD>(d, p, sh, t, buf);
    __syncthreads();  // buf is refilled by the next iteration's copies
    s = s + 1 == K ? 0 : s + 1;
  }
  cp_async_wait<0>();
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
