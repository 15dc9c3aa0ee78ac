// Per-cell fused step with single-buffer AA-pattern streaming.
//
// One array A[a][cell] holds all populations.  With step counter n:
//   n even: A[a][x] = f_a^n(x)               (canonical, pre-collision)
//   n odd:  A[abar][x] = f*_a^{n-1}(x)       (post-collision of step n-1,
//                                              kept in the cell it left)
// Even step:  read A[a][x] for all a, collide, write f*_a to A[abar][x].
// Odd step:   read f_a(x) from A[abar][x - c_a], collide, write f*_a to
//             A[a][x + c_a]; the cell reads and writes exactly the same
//             2Q locations, so the in-place update is race-free.
// Halfway bounce-back (the wall midway between a fluid node and the ghost
// node beyond it): in the odd step a link whose source x - c_a is a ghost
// reads the cell's own A[a][x] (its reflected post-collision population)
// plus 6 w_a (c_a . u_wall), and a link whose target x + c_a is a ghost
// writes the reflected value f*_a - 6 w_a (c_a . u_wall) to A[abar][x], i.e.
// straight into its canonical slot.  The even step touches no neighbour.
// Each update therefore moves exactly 2Q stored values.
#pragma once

#include "lbm_model.cuh"

namespace lbm {

template <typename R>
struct Domain {
  void* f;           // population buffer, Q*N values of the storage type
  int nx, ny, nz;
  int64_t N;         // nx*ny*nz
  int per[3];        // axis is periodic
  int moving;        // bit f set: face f is a moving wall
  R uw[6][3];        // velocity of each face (zero unless MOVING_WALL)
  Rates<R> s;
  R F[3];            // body force at the step's time level t_n
};

// Node (x,y,z)+(dx,dy,dz) with dx,dy,dz in {-1,0,1}.  Returns true and its
// cell index if it is a fluid node (after periodic wrap); otherwise false
// and, in `beyond`, the faces (bit f = face f) the ghost node lies beyond.
template <typename R>
__host__ __device__ __forceinline__ bool resolve(const Domain<R>& d, int x, int y, int z,
                                        int dx, int dy, int dz, int64_t& j,
                                        int& beyond) {
  beyond = 0;
  int v[3] = {x + dx, y + dy, z + dz};
  const int n[3] = {d.nx, d.ny, d.nz};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (v[k] < 0) {
      if (d.per[k]) v[k] += n[k];
      else beyond |= 1 << (2 * k);
    } else if (v[k] >= n[k]) {
      if (d.per[k]) v[k] -= n[k];
      else beyond |= 1 << (2 * k + 1);
    }
  }
  j = (int64_t)v[0] + (int64_t)d.nx * ((int64_t)v[1] + (int64_t)d.ny * v[2]);
  return beyond == 0;
}

// c . u_wall for a ghost node beyond the faces in `beyond`: the first
// moving face in x-, x+, y-, y+, z-, z+ order wins (edge and corner ghosts of
// a lid layer belong to the lid).
template <typename R>
__host__ __device__ __forceinline__ R ghost_dot(const Domain<R>& d, int beyond, int cx,
                                       int cy, int cz) {
  const int hit = beyond & d.moving;
  if (!hit) return R(0);
#pragma unroll
  for (int face = 0; face < 6; ++face)
    if ((hit >> face) & 1)
      return R(cx) * d.uw[face][0] + R(cy) * d.uw[face][1] + R(cz) * d.uw[face][2];
  return R(0);
}

// Pre-collision populations f^n of cell (x,y,z) (index i) into fv.
template <int Q, typename S, typename R, bool ODD>
__host__ __device__ __forceinline__ void gather(const Domain<R>& d, const S* __restrict__ f,
                                       int x, int y, int z, int64_t i,
                                       bool interior, R* fv) {
  const int64_t N = d.N;
  if constexpr (!ODD) {
    [&]<int... A>(std::integer_sequence<int, A...>) {
      ((fv[A] = Codec<S, R>::load(f + A * N + i)), ...);
    }(std::make_integer_sequence<int, Q>{});
  } else if (interior) {
    const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
    [&]<int... A>(std::integer_sequence<int, A...>) {
      ((fv[A] = Codec<S, R>::load(
            f + opposite<Q>(A) * N + i -
            (Lattice<Q>::c(A, 0) + Lattice<Q>::c(A, 1) * sy +
             Lattice<Q>::c(A, 2) * sz))),
       ...);
    }(std::make_integer_sequence<int, Q>{});
  } else {
    [&]<int... A>(std::integer_sequence<int, A...>) {
      (
          [&] {
            constexpr int cx = Lattice<Q>::c(A, 0), cy = Lattice<Q>::c(A, 1),
                          cz = Lattice<Q>::c(A, 2);
            int64_t j;
            int beyond;
            if (resolve(d, x, y, z, -cx, -cy, -cz, j, beyond)) {
              fv[A] = Codec<S, R>::load(f + opposite<Q>(A) * N + j);
            } else {
              fv[A] = Codec<S, R>::load(f + A * N + i) +
                      R(6.0 * Lattice<Q>::w(A)) * ghost_dot(d, beyond, cx, cy, cz);
            }
          }(),
          ...);
    }(std::make_integer_sequence<int, Q>{});
  }
}

// Post-collision populations f* of cell (x,y,z) from fv into storage.
template <int Q, typename S, typename R, bool ODD>
__host__ __device__ __forceinline__ void scatter(const Domain<R>& d, S* __restrict__ f,
                                        int x, int y, int z, int64_t i,
                                        bool interior, const R* fv) {
  const int64_t N = d.N;
  if constexpr (!ODD) {
    [&]<int... A>(std::integer_sequence<int, A...>) {
      ((Codec<S, R>::store(f + opposite<Q>(A) * N + i, fv[A])), ...);
    }(std::make_integer_sequence<int, Q>{});
  } else if (interior) {
    const int64_t sy = d.nx, sz = (int64_t)d.nx * d.ny;
    [&]<int... A>(std::integer_sequence<int, A...>) {
      ((Codec<S, R>::store(f + A * N + i +
                               (Lattice<Q>::c(A, 0) + Lattice<Q>::c(A, 1) * sy +
                                Lattice<Q>::c(A, 2) * sz),
                           fv[A])),
       ...);
    }(std::make_integer_sequence<int, Q>{});
  } else {
    [&]<int... A>(std::integer_sequence<int, A...>) {
      (
          [&] {
            constexpr int cx = Lattice<Q>::c(A, 0), cy = Lattice<Q>::c(A, 1),
                          cz = Lattice<Q>::c(A, 2);
            int64_t j;
            int beyond;
            if (resolve(d, x, y, z, cx, cy, cz, j, beyond)) {
              Codec<S, R>::store(f + A * N + j, fv[A]);
            } else {
              Codec<S, R>::store(
                  f + opposite<Q>(A) * N + i,
                  fv[A] - R(6.0 * Lattice<Q>::w(A)) * ghost_dot(d, beyond, cx, cy, cz));
            }
          }(),
          ...);
    }(std::make_integer_sequence<int, Q>{});
  }
}

template <typename R>
__host__ __device__ __forceinline__ bool is_interior(const Domain<R>& d, int x, int y, int z) {
  return x > 0 && x < d.nx - 1 && y > 0 && y < d.ny - 1 && z > 0 && z < d.nz - 1;
}

// The whole fused update of one cell: gather (stream), collide, scatter.
template <int Q, typename S, typename R, bool ODD, bool FORCE>
__host__ __device__ __forceinline__ void update_cell(const Domain<R>& d, S* __restrict__ f,
                                            int x, int y, int z) {
  const int64_t i = (int64_t)x + (int64_t)d.nx * ((int64_t)y + (int64_t)d.ny * z);
  const bool interior = ODD ? is_interior(d, x, y, z) : true;
  R fv[Q];
  gather<Q, S, R, ODD>(d, f, x, y, z, i, interior, fv);
  R ux, uy, uz;
  collide<Q, FORCE>(fv, d.s, d.F[0], d.F[1], d.F[2], ux, uy, uz);
  scatter<Q, S, R, ODD>(d, f, x, y, z, i, interior, fv);
}

// Inverse of gather: put canonical pre-collision values fv of cell (x,y,z)
// where the current parity keeps them (checkpoint restore / init).
template <int Q, typename S, typename R, bool ODD>
__host__ __device__ __forceinline__ void put_canonical(const Domain<R>& d, S* __restrict__ f,
                                              int x, int y, int z, int64_t i,
                                              const R* fv) {
  const int64_t N = d.N;
  [&]<int... A>(std::integer_sequence<int, A...>) {
    (
        [&] {
          if constexpr (!ODD) {
            Codec<S, R>::store(f + A * N + i, fv[A]);
          } else {
            constexpr int cx = Lattice<Q>::c(A, 0), cy = Lattice<Q>::c(A, 1),
                          cz = Lattice<Q>::c(A, 2);
            int64_t j;
            int beyond;
            if (resolve(d, x, y, z, -cx, -cy, -cz, j, beyond)) {
              Codec<S, R>::store(f + opposite<Q>(A) * N + j, fv[A]);
            } else {
              Codec<S, R>::store(
                  f + A * N + i,
                  fv[A] - R(6.0 * Lattice<Q>::w(A)) * ghost_dot(d, beyond, cx, cy, cz));
            }
          }
        }(),
        ...);
  }(std::make_integer_sequence<int, Q>{});
}

}  // namespace lbm
