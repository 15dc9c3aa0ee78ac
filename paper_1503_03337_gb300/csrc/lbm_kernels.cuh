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

#include "lbm_collide.cuh"

namespace lbm {

template <typename R>
struct Domain {
  void* f;           // population buffer, Q*N values of the storage type
  int nx, ny, nz;
  int64_t N;         // nx*ny*nz
  int per[3];        // axis is periodic
  int moving;        // bit f set: face f is a moving wall
  int sym;           // bit f set: face f is a symmetry (free-slip) plane
  R uw[6][3];        // velocity of each face (zero unless MOVING_WALL)
  // Edge profile of a moving face f (the lid corner velocities of Sec.
  // 4.3): with edge_axis[f] = k + 1, a cell in the first (last) node column
  // along axis k sees uw[f] * edge_scale[f][0] ([1]); a one-node axis takes
  // [0]; edge_axis[f] = 0: uniform.
  int edge_axis[6];
  R edge_scale[6][2];
  Rates<R> s;
  R F[3];            // body force at the step's time level t_n
  uint32_t key;      // per-step key of the stochastic-rounding hash
  // Solid nodes (general geometry), null if none: per cell, bit a set if
  // the pull source x - c_a (after periodic wraps and symmetry mirrors; not
  // beyond a wall) is a solid node, so that link bounces back off a wall at
  // rest; kSolidCell marks a solid cell itself, which no step updates.
  const uint32_t* solid;
  // Element offsets from a cell's slot 0 (index i) used by interior cells
  // on odd steps:
  //   pull[a] = abar*N - s(c_a)     (where f_a(x) is read)
  //   push[a] = a*N + s(c_a)        (where f*_a(x) is written)
  // with s(c) = cx + cy*nx + cz*nx*ny.  Filled by fill_offsets().  pull and
  // push hold them while Q*N < 2^31; pull64 / push64 always, for the wide
  // kernels of larger domains (cell indices stay 32-bit: N < 2^31).
  int pull[26], push[26];
  int64_t pull64[26], push64[26];
};

// Index type of population offsets a*N + i: 32-bit while Q*N < 2^31, else
// 64-bit (the WIDE kernel variants).
template <bool WIDE>
using PopIndex = std::conditional_t<WIDE, int64_t, int>;

template <bool WIDE, typename R>
__host__ __device__ __forceinline__ PopIndex<WIDE> pull_offset(const Domain<R>& d, int a) {
  if constexpr (WIDE) return d.pull64[a];
  else return d.pull[a];
}
template <bool WIDE, typename R>
__host__ __device__ __forceinline__ PopIndex<WIDE> push_offset(const Domain<R>& d, int a) {
  if constexpr (WIDE) return d.push64[a];
  else return d.push[a];
}

constexpr uint32_t kSolidCell = 0x80000000u;

// Domain::solid word of cell i from the byte mask of solid nodes (nonzero =
// solid): kSolidCell for a solid cell, else bit a set when the pull source
// x - c_a -- wrapped across periodic axes (bit k of `per`), mirrored across
// symmetry faces (bit f of `sym`), and not beyond a wall -- is solid.
template <int Q>
__host__ __device__ inline uint32_t solid_link_bits(int nx, int ny, int nz, int per, int sym,
                                                    const uint8_t* bytes, int64_t i) {
  if (bytes[i]) return kSolidCell;
  const int n[3] = {nx, ny, nz};
  const int xyz[3] = {(int)(i % nx), (int)((i / nx) % ny), (int)(i / ((int64_t)nx * ny))};
  uint32_t m = 0;
  for (int a = 0; a < Q; ++a) {
    int src[3];
    bool beyond_wall = false;
    for (int k = 0; k < 3; ++k) {
      int v = xyz[k] - Lattice<Q>::c(a, k);
      if (v < 0 || v >= n[k]) {
        const int face = v < 0 ? 2 * k : 2 * k + 1;
        if ((per >> k) & 1) v += v < 0 ? n[k] : -n[k];
        else if ((sym >> face) & 1) v = xyz[k];
        else beyond_wall = true;
      }
      src[k] = v;
    }
    if (!beyond_wall && bytes[src[0] + (int64_t)nx * (src[1] + (int64_t)ny * src[2])])
      m |= 1u << a;
  }
  return m;
}

// Per-step key of the stochastic-rounding hash.
__host__ __device__ inline uint32_t step_key(int64_t n) {
  return mix32(0x5eedu ^ (uint32_t(n) * 0x632be5abu) ^ uint32_t(uint64_t(n) >> 32));
}

template <int Q, typename R>
__host__ __device__ inline void fill_offsets(Domain<R>& d) {
  const int64_t N = d.N, sy = d.nx, sz = (int64_t)d.nx * d.ny;
  for (int a = 0; a < Q; ++a) {
    const int64_t s = Lattice<Q>::c(a, 0) + Lattice<Q>::c(a, 1) * sy + Lattice<Q>::c(a, 2) * sz;
    d.pull64[a] = opposite<Q>(a) * N - s;
    d.push64[a] = a * N + s;
    d.pull[a] = (int)d.pull64[a];  // exact while Q*N < 2^31
    d.push[a] = (int)d.push64[a];
  }
}

// Edge-profile factor of moving face `face` for a cell whose position bits
// are `edge` (bit 2k: first node column along axis k; bit 2k+1: last, and
// not first).
template <typename R>
__host__ __device__ __forceinline__ R edge_factor(const Domain<R>& d, int face, int edge) {
  const int k = d.edge_axis[face] - 1;
  if (k < 0) return R(1);
  if ((edge >> (2 * k)) & 1) return d.edge_scale[face][0];
  if ((edge >> (2 * k + 1)) & 1) return d.edge_scale[face][1];
  return R(1);
}

// c . u_wall for a ghost node beyond the faces in `beyond`, seen from a cell
// with position bits `edge`: the first moving face in x-, x+, y-, y+, z-,
// z+ order wins (edge and corner ghosts of a lid layer belong to the lid).
template <typename R>
__host__ __device__ __forceinline__ R ghost_dot(const Domain<R>& d, int edge, int beyond,
                                                int cx, int cy, int cz) {
  const int hit = beyond & d.moving;
  if (!hit) return R(0);
#pragma unroll
  for (int face = 0; face < 6; ++face)
    if ((hit >> face) & 1) {
      const R e = edge_factor(d, face, edge);
      return R(cx) * (d.uw[face][0] * e) + R(cy) * (d.uw[face][1] * e) +
             R(cz) * (d.uw[face][2] * e);
    }
  return R(0);
}

// Neighbour addressing of one cell for the odd (neighbour-touching) step.
// Along each axis: the index offset to the -1 / +1 neighbour (periodic wrap
// applied; 0 if that neighbour is a ghost node) and whether it is a ghost
// node beyond a wall.  Computed once per cell; each link then costs a few
// integer adds and one select, with no divergent branch.
// Beyond a symmetry face the ghost mirrors the node across the halfway
// plane: along that axis the neighbour is the node itself (offset 0) and the
// population is the mirror one (flag sm / sp).  A link that also crosses a
// wall on another axis is a wall link (gm / gp win).
struct Links {
  int om[3], op[3];
  bool gm[3], gp[3];  // ghost beyond a wall
  bool sm[3], sp[3];  // ghost beyond a symmetry face
  int edge;           // position bits of the cell (see edge_factor)
  bool interior;  // every neighbour is a fluid, unwrapped node: use pull/push
  uint32_t solid;     // bit a: the pull source of link a is a solid node
};

__host__ __device__ __forceinline__ int edge_bits(int v, int n, int k) {
  return v == 0 ? 1 << (2 * k) : (v == n - 1 ? 2 << (2 * k) : 0);
}

template <typename R>
__host__ __device__ __forceinline__ void axis_links(int v, int n, int stride, int per,
                                                    int sym_lo, int sym_hi, int& om, int& op,
                                                    bool& gm, bool& gp, bool& sm, bool& sp) {
  const bool lo = v == 0, hi = v == n - 1;
  om = !lo ? -stride : (per ? (n - 1) * stride : 0);
  op = !hi ? stride : (per ? -(n - 1) * stride : 0);
  sm = lo && !per && sym_lo;
  sp = hi && !per && sym_hi;
  gm = lo && !per && !sym_lo;
  gp = hi && !per && !sym_hi;
}

template <typename R>
__host__ __device__ __forceinline__ Links make_links(const Domain<R>& d, int x, int y, int z) {
  Links L;
  const int sy = d.nx, sz = d.nx * d.ny;
  axis_links<R>(x, d.nx, 1, d.per[0], d.sym & 1, (d.sym >> 1) & 1, L.om[0], L.op[0], L.gm[0],
                L.gp[0], L.sm[0], L.sp[0]);
  axis_links<R>(y, d.ny, sy, d.per[1], (d.sym >> 2) & 1, (d.sym >> 3) & 1, L.om[1], L.op[1],
                L.gm[1], L.gp[1], L.sm[1], L.sp[1]);
  axis_links<R>(z, d.nz, sz, d.per[2], (d.sym >> 4) & 1, (d.sym >> 5) & 1, L.om[2], L.op[2],
                L.gm[2], L.gp[2], L.sm[2], L.sp[2]);
  L.edge = edge_bits(x, d.nx, 0) | edge_bits(y, d.ny, 1) | edge_bits(z, d.nz, 2);
  L.interior = false;
  L.solid = d.solid ? d.solid[x + (int64_t)d.nx * (y + (int64_t)d.ny * z)] : 0u;
  return L;
}

// Links of a cell whose neighbours are all fluid and unwrapped.
template <typename R>
__host__ __device__ __forceinline__ Links make_links_interior(const Domain<R>& d) {
  Links L;
  const int sy = d.nx, sz = d.nx * d.ny;
  L.om[0] = -1;
  L.op[0] = 1;
  L.om[1] = -sy;
  L.op[1] = sy;
  L.om[2] = -sz;
  L.op[2] = sz;
  L.gm[0] = L.gp[0] = L.gm[1] = L.gp[1] = L.gm[2] = L.gp[2] = false;
  L.sm[0] = L.sp[0] = L.sm[1] = L.sp[1] = L.sm[2] = L.sp[2] = false;
  L.edge = 0;
  L.interior = true;
  L.solid = 0u;
  return L;
}

// Links of a cell whose y and z neighbours are all fluid and unwrapped (the
// bulk of a box): only x needs the select.
template <typename R>
__host__ __device__ __forceinline__ Links make_links_x(const Domain<R>& d, int x) {
  Links L;
  const int sy = d.nx, sz = d.nx * d.ny;
  axis_links<R>(x, d.nx, 1, d.per[0], d.sym & 1, (d.sym >> 1) & 1, L.om[0], L.op[0], L.gm[0],
                L.gp[0], L.sm[0], L.sp[0]);
  L.sm[1] = L.sp[1] = L.sm[2] = L.sp[2] = false;
  L.edge = edge_bits(x, d.nx, 0);
  L.om[1] = -sy;
  L.op[1] = sy;
  L.om[2] = -sz;
  L.op[2] = sz;
  L.gm[1] = L.gp[1] = L.gm[2] = L.gp[2] = false;
  L.interior = false;
  L.solid = 0u;
  return L;
}

// Offset, wall-ghost flag and mirror axes (bit k: the link crosses a
// symmetry face normal to axis k) of the node x + s*c_A (s = -1: pull
// source, +1: push target).  SYM = false: the domain has no symmetry face
// (mirror stays 0 and the mirrored indexing folds away).
template <int Q, int A, int SIGN, bool SYM = true, bool SOLID = true>
__host__ __device__ __forceinline__ void link_of(const Links& L, int& off, bool& ghost,
                                                 int& mirror) {
  off = 0;
  ghost = false;
  mirror = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int c = SIGN * Lattice<Q>::c(A, k);
    if (c < 0) {
      off += L.om[k];
      ghost = ghost || L.gm[k];
      if (SYM && L.sm[k]) mirror |= 1 << k;
    } else if (c > 0) {
      off += L.op[k];
      ghost = ghost || L.gp[k];
      if (SYM && L.sp[k]) mirror |= 1 << k;
    }
  }
  // a solid pull source (SIGN -1: x - c_A) or push target (x + c_A, the
  // pull source of the opposite link): bounce-back at rest.  SOLID = false:
  // the caller knows L.solid is zero.
  if (SOLID && ((L.solid >> (SIGN < 0 ? A : opposite<Q>(A))) & 1u)) ghost = true;
}

// The population whose velocity is c_A with the components of the axes in
// `mask` reversed (every lattice here is closed under axis reflections).
template <int Q>
__host__ __device__ constexpr int mirror_of(int a, int mask) {
  int c[3];
  for (int k = 0; k < 3; ++k) c[k] = (mask >> k) & 1 ? -Lattice<Q>::c(a, k) : Lattice<Q>::c(a, k);
  for (int b = 0; b < Q; ++b)
    if (Lattice<Q>::c(b, 0) == c[0] && Lattice<Q>::c(b, 1) == c[1] && Lattice<Q>::c(b, 2) == c[2])
      return b;
  return -1;
}
template <int Q>
__host__ __device__ constexpr bool mirrors_closed() {
  for (int a = 0; a < Q; ++a)
    for (int m = 0; m < 8; ++m)
      if (mirror_of<Q>(a, m) < 0) return false;
  return true;
}
static_assert(mirrors_closed<14>() && mirrors_closed<18>() && mirrors_closed<26>(),
              "lattice not closed under mirrors");

// mirror_of<Q>(A, mask) for a runtime mask (a select among eight constants)
template <int Q, int A>
__host__ __device__ __forceinline__ int mirror_rt(int mask) {
  switch (mask) {
    case 1: return mirror_of<Q>(A, 1);
    case 2: return mirror_of<Q>(A, 2);
    case 3: return mirror_of<Q>(A, 3);
    case 4: return mirror_of<Q>(A, 4);
    case 5: return mirror_of<Q>(A, 5);
    case 6: return mirror_of<Q>(A, 6);
    case 7: return mirror_of<Q>(A, 7);
    default: return A;
  }
}
template <int Q, int A>
__host__ __device__ __forceinline__ int opposite_mirror_rt(int mask) {
  switch (mask) {
    case 1: return opposite<Q>(mirror_of<Q>(A, 1));
    case 2: return opposite<Q>(mirror_of<Q>(A, 2));
    case 3: return opposite<Q>(mirror_of<Q>(A, 3));
    case 4: return opposite<Q>(mirror_of<Q>(A, 4));
    case 5: return opposite<Q>(mirror_of<Q>(A, 5));
    case 6: return opposite<Q>(mirror_of<Q>(A, 6));
    case 7: return opposite<Q>(mirror_of<Q>(A, 7));
    default: return opposite<Q>(A);
  }
}

// The ghost node beyond the faces this link crosses: bit mask of those faces.
template <int Q, int A, int SIGN>
__host__ __device__ __forceinline__ int link_faces(const Links& L) {
  int m = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int c = SIGN * Lattice<Q>::c(A, k);
    if (c < 0 && L.gm[k]) m |= 1 << (2 * k);
    if (c > 0 && L.gp[k]) m |= 1 << (2 * k + 1);
  }
  return m;
}

// Does the cell touch a moving face (so some link needs the wall term)?
template <typename R>
__host__ __device__ __forceinline__ bool touches_moving(const Domain<R>& d, const Links& L) {
  const int m = (L.gm[0] ? 1 : 0) | (L.gp[0] ? 2 : 0) | (L.gm[1] ? 4 : 0) |
                (L.gp[1] ? 8 : 0) | (L.gm[2] ? 16 : 0) | (L.gp[2] ? 32 : 0);
  return (m & d.moving) != 0;
}

// Moving-wall terms of the links of a pull whose source node is a ghost
// beyond a moving face: +6 w_a (c_a . u_w) (halfway bounce-back off a moving
// wall).
template <int Q, typename R>
__host__ __device__ __forceinline__ void add_pull_wall_terms(const Domain<R>& d, const Links& L,
                                                             R* fv) {
  if (d.moving && touches_moving(d, L)) {
    [&]<int... A>(std::integer_sequence<int, A...>) {
      (
          [&] {
            const int faces = link_faces<Q, A, -1>(L);
            if (faces)
              fv[A] += R(6.0 * Lattice<Q>::w(A)) *
                       ghost_dot(d, L.edge, faces, Lattice<Q>::c(A, 0), Lattice<Q>::c(A, 1),
                                 Lattice<Q>::c(A, 2));
          }(),
          ...);
    }(std::make_integer_sequence<int, Q>{});
  }
}

// Pre-collision populations f^n of cell i into fv (CG: L2-only loads; SYM:
// the domain may have symmetry faces).
template <int Q, typename S, typename R, bool ODD, bool CG = false, bool SYM = true,
          bool SOLID = true, bool WIDE = false>
__host__ __device__ __forceinline__ void gather(const Domain<R>& d, const S* __restrict__ f,
                                                int i, const Links& L, R* fv) {
  using Ix = PopIndex<WIDE>;
  const Ix N = (Ix)d.N;
  const S* __restrict__ fc = f + i;
  if constexpr (!ODD) {
    [&]<int... A>(std::integer_sequence<int, A...>) {
      ((fv[A] = load_pop<S, R, CG>(fc + (size_t)A * d.N)), ...);
    }(std::make_integer_sequence<int, Q>{});
  } else if (L.interior) {
    [&]<int... A>(std::integer_sequence<int, A...>) {
      ((fv[A] = load_pop<S, R, CG>(fc + pull_offset<WIDE>(d, A))), ...);
    }(std::make_integer_sequence<int, Q>{});
  } else {
    // f_a(x) = A[abar][x - c_a], or A[a][x] if x - c_a is a wall ghost;
    // beyond a symmetry face the source is the mirror node and population
    [&]<int... A>(std::integer_sequence<int, A...>) {
      (
          [&] {
            int off, mirror;
            bool ghost;
            link_of<Q, A, -1, SYM, SOLID>(L, off, ghost, mirror);
            const Ix idx =
                ghost ? (A * N + i) : (opposite_mirror_rt<Q, A>(mirror) * N + i + off);
            fv[A] = load_pop<S, R, CG>(f + idx);
          }(),
          ...);
    }(std::make_integer_sequence<int, Q>{});
    add_pull_wall_terms<Q>(d, L, fv);
  }
}

// Random bits of the stochastic rounding.  Cell i and the step's key give
// one hash per cell, sr_cell_hash; the direction pair (2K, 2K+1) of the cell
// draws the 32 bits sr_bits<K>(hash), whose low half rounds direction 2K and
// whose high half rounds 2K+1 (the halves a two-value conversion takes from
// its random operand).  The bits therefore belong to (cell, direction, step)
// alone, whether a cell is stored by itself or as one half of an x-adjacent
// pair.
__host__ __device__ __forceinline__ uint32_t sr_cell_hash(int i, uint32_t key) {
  return mix32(uint32_t(i) ^ key);
}
template <int K>
__host__ __device__ __forceinline__ uint32_t sr_bits(uint32_t h) {
  return mix32_short(h + uint32_t(K + 1) * 0x9e3779b9u);
}

template <typename S>
__host__ __device__ __forceinline__ void store_half(S* p, uint16_t v) {
#ifdef __CUDA_ARCH__
  *reinterpret_cast<unsigned short*>(p) = v;
#else
  memcpy(p, &v, 2);
#endif
}

// Store the Q post-collision values fv of one cell at the addresses
// addr.operator()<A>() (stochastically rounded in direction pairs if SR, h =
// sr_cell_hash of the cell).
template <int Q, typename S, typename R, bool SR, typename Addr>
__host__ __device__ __forceinline__ void store_cell(const R* fv, uint32_t h, Addr&& addr) {
  if constexpr (SR) {
    [&]<int... K>(std::integer_sequence<int, K...>) {
      (
          [&] {
            const uint32_t w =
                Stochastic<S>::pack2(float(fv[2 * K + 1]), float(fv[2 * K]), sr_bits<K>(h));
            store_half(addr.template operator()<2 * K>(), uint16_t(w & 0xffffu));
            store_half(addr.template operator()<2 * K + 1>(), uint16_t(w >> 16));
          }(),
          ...);
    }(std::make_integer_sequence<int, Q / 2>{});
  } else {
    [&]<int... A>(std::integer_sequence<int, A...>) {
      (Codec<S, R>::store(addr.template operator()<A>(), fv[A]), ...);
    }(std::make_integer_sequence<int, Q>{});
  }
}

// Post-collision populations f* of cell i from fv into storage (`key`: the
// step's stochastic-rounding key; SYM as in gather).
template <int Q, typename S, typename R, bool ODD, bool SR = false, bool SYM = true,
          bool SOLID = true, bool WIDE = false>
__host__ __device__ __forceinline__ void scatter(const Domain<R>& d, S* __restrict__ f,
                                                 int i, const Links& L, R* fv, uint32_t key) {
  using Ix = PopIndex<WIDE>;
  const Ix N = (Ix)d.N;
  const uint32_t h = SR ? sr_cell_hash(i, key) : 0u;
  S* __restrict__ fc = f + i;
  if constexpr (!ODD) {
    store_cell<Q, S, R, SR>(fv, h, [&]<int A>() { return fc + (size_t)opposite<Q>(A) * d.N; });
  } else if (L.interior) {
    store_cell<Q, S, R, SR>(fv, h, [&]<int A>() { return fc + push_offset<WIDE>(d, A); });
  } else {
    if (d.moving && touches_moving(d, L)) {
      [&]<int... A>(std::integer_sequence<int, A...>) {
        (
            [&] {
              const int faces = link_faces<Q, A, 1>(L);
              if (faces)
                fv[A] -= R(6.0 * Lattice<Q>::w(A)) *
                         ghost_dot(d, L.edge, faces, Lattice<Q>::c(A, 0), Lattice<Q>::c(A, 1),
                                   Lattice<Q>::c(A, 2));
            }(),
            ...);
      }(std::make_integer_sequence<int, Q>{});
    }
    // f*_a goes to A[a][x + c_a], or back into A[abar][x] if x + c_a is a
    // wall ghost; beyond a symmetry face it becomes the mirror population of
    // the mirror node (the slot this cell's mirrored pull reads)
    store_cell<Q, S, R, SR>(fv, h, [&]<int A>() {
      int off, mirror;
      bool ghost;
      link_of<Q, A, 1, SYM, SOLID>(L, off, ghost, mirror);
      const Ix idx = ghost ? (opposite<Q>(A) * N + i) : (mirror_rt<Q, A>(mirror) * N + i + off);
      return f + idx;
    });
  }
}

template <int Q, typename S, typename R, bool ODD, bool FORCE, bool SR, bool CG = false,
          bool SYM = true, bool SOLID = false, bool WIDE = false>
__host__ __device__ __forceinline__ void update_with_links(const Domain<R>& d,
                                                           S* __restrict__ f, int i,
                                                           const Links& L, const R* F,
                                                           const uint32_t* key) {
  R fv[Q];
  gather<Q, S, R, ODD, CG, SYM, SOLID, WIDE>(d, f, i, L, fv);
  R ux, uy, uz;
  collide<Q, FORCE>(fv, d.s, F[0], F[1], F[2], ux, uy, uz);
  scatter<Q, S, R, ODD, SR, SYM, SOLID, WIDE>(d, f, i, L, fv, SR ? *key : 0u);
}

// Does any active lane of the warp hold a nonzero v (every lane on the
// host, where cells run one at a time)?
__host__ __device__ __forceinline__ bool warp_any(bool v) {
#ifdef __CUDA_ARCH__
  return __any_sync(__activemask(), v);
#else
  return v;
#endif
}

// The whole fused update of one cell: gather (stream), collide, scatter.
// Odd steps pick one of three addressing variants.  `x_lo`..`x_hi` is the
// x-range of the calling warp: when a warp lies within one x-row (block
// width a multiple of 32) every test below is uniform across the warp, so
// the variants never diverge inside a warp.  The two boundary variants come
// with and without the mirrored links of symmetry faces (d.sym is uniform
// across the grid), so domains without one pay nothing for them.
// update_cell_at reads the step's body force F[0..2] and rounding key *key
// where they are used (F and key may live outside the descriptor);
// update_cell takes them from the descriptor.
template <int Q, typename S, typename R, bool ODD, bool FORCE, bool SR = false,
          bool CG = false, bool WIDE = false>
__host__ __device__ __forceinline__ void update_cell_at(const Domain<R>& d, S* __restrict__ f,
                                                        const R* F, const uint32_t* key, int x,
                                                        int y, int z, int x_lo, int x_hi) {
  const int i = x + d.nx * (y + d.ny * z);
  if constexpr (!ODD) {
    if (d.solid && (d.solid[i] & kSolidCell)) return;  // solid cells hold no flow
    Links L{};
    update_with_links<Q, S, R, false, FORCE, SR, CG, true, false, WIDE>(d, f, i, L, F, key);
  } else {
    if (d.solid) {
      // a warp with any solid-touching link takes the full addressing with
      // the cells' solid bits (the vote comes before any lane leaves)
      const uint32_t sm = d.solid[i];
      if (warp_any(sm != 0u)) {
        if (sm & kSolidCell) return;
        if (d.sym)
          update_with_links<Q, S, R, true, FORCE, SR, CG, true, true, WIDE>(
              d, f, i, make_links(d, x, y, z), F, key);
        else
          update_with_links<Q, S, R, true, FORCE, SR, CG, false, true, WIDE>(
              d, f, i, make_links(d, x, y, z), F, key);
        return;
      }
    }
    if (y > 0 && y < d.ny - 1 && z > 0 && z < d.nz - 1) {
      if (x_lo > 0 && x_hi < d.nx - 1)
        update_with_links<Q, S, R, true, FORCE, SR, CG, true, false, WIDE>(d, f, i, make_links_interior(d), F,
                                                        key);
      else if (d.sym)
        update_with_links<Q, S, R, true, FORCE, SR, CG, true, false, WIDE>(d, f, i, make_links_x(d, x), F,
                                                              key);
      else
        update_with_links<Q, S, R, true, FORCE, SR, CG, false, false, WIDE>(d, f, i, make_links_x(d, x), F,
                                                               key);
    } else if (d.sym) {
      update_with_links<Q, S, R, true, FORCE, SR, CG, true, false, WIDE>(d, f, i, make_links(d, x, y, z), F,
                                                            key);
    } else {
      update_with_links<Q, S, R, true, FORCE, SR, CG, false, false, WIDE>(d, f, i, make_links(d, x, y, z), F,
                                                             key);
    }
  }
}

template <int Q, typename S, typename R, bool ODD, bool FORCE, bool SR = false,
          bool CG = false, bool WIDE = false>
__host__ __device__ __forceinline__ void update_cell(const Domain<R>& d, S* __restrict__ f,
                                                     int x, int y, int z, int x_lo = -1,
                                                     int x_hi = -1) {
  update_cell_at<Q, S, R, ODD, FORCE, SR, CG, WIDE>(d, f, d.F, &d.key, x, y, z, x_lo, x_hi);
}

// Two storage values of x-adjacent cells as one word (8 bytes for FP32,
// 4 bytes for FP16 / BF16), unpacked to and packed from a pf2.
template <typename S>
struct Pair2;
template <>
struct Pair2<float> {
  using type = float2;
  __device__ static pf2 unpack(float2 v) { return pf2(v.x, v.y); }
  __device__ static float2 pack(pf2 v) { return v.v; }
};
template <>
struct Pair2<__half> {
  using type = __half2;
  __device__ static pf2 unpack(__half2 v) {
    const float2 t = __half22float2(v);
    return pf2(t.x, t.y);
  }
  __device__ static __half2 pack(pf2 v) { return __floats2half2_rn(v.v.x, v.v.y); }
};
template <>
struct Pair2<__nv_bfloat16> {
  using type = __nv_bfloat162;
  __device__ static pf2 unpack(__nv_bfloat162 v) {
    const float2 t = __bfloat1622float2(v);
    return pf2(t.x, t.y);
  }
  __device__ static __nv_bfloat162 pack(pf2 v) { return __floats2bfloat162_rn(v.v.x, v.v.y); }
};

// Even step of the two x-adjacent cells i, i + 1 (i even): each population
// of the pair is one load and one store of a two-value word, so a warp's
// access covers twice the bytes of one cell per thread (128 bytes for FP16
// / BF16 storage, which one value per thread leaves at 64), and the two
// cells collide together in packed FP32x2.  Needs nx even (then N is even
// and a pair never straddles a row).  An even step touches only the cell's
// own slots, so no links are needed.  SR: each word is one stochastic pair
// conversion with the random bits the one-cell update uses for both cells.
template <int Q, typename S, bool FORCE, bool SR = false>
__device__ __forceinline__ void update_pair_even(const Domain<float>& d, S* __restrict__ f,
                                                 int i) {
  using W = typename Pair2<S>::type;
  W* __restrict__ g = reinterpret_cast<W*>(f);
  const int M = (int)(d.N >> 1), j = i >> 1;
  pf2 fv[Q];
  [&]<int... A>(std::integer_sequence<int, A...>) {
    ((fv[A] = Pair2<S>::unpack(g[j + A * M])), ...);
  }(std::make_integer_sequence<int, Q>{});
  pf2 ux, uy, uz;
  collide<Q, FORCE>(fv, d.s, d.F[0], d.F[1], d.F[2], ux, uy, uz);
  if constexpr (SR) {
    // random bits of direction A for cells i (low half of the operand) and
    // i + 1 (high half): the halves of sr_bits<A/2> of each cell's hash that
    // round direction A
    const uint32_t he = sr_cell_hash(i, d.key), ho = sr_cell_hash(i + 1, d.key);
    uint32_t* __restrict__ g32 = reinterpret_cast<uint32_t*>(f);
    [&]<int... K>(std::integer_sequence<int, K...>) {
      (
          [&] {
            const uint32_t re = sr_bits<K>(he), ro = sr_bits<K>(ho);
            g32[j + opposite<Q>(2 * K) * M] =
                Stochastic<S>::pack2(fv[2 * K].v.y, fv[2 * K].v.x, (re & 0xffffu) | (ro << 16));
            g32[j + opposite<Q>(2 * K + 1) * M] = Stochastic<S>::pack2(
                fv[2 * K + 1].v.y, fv[2 * K + 1].v.x, (re >> 16) | (ro & 0xffff0000u));
          }(),
          ...);
    }(std::make_integer_sequence<int, Q / 2>{});
  } else {
    [&]<int... A>(std::integer_sequence<int, A...>) {
      ((g[j + opposite<Q>(A) * M] = Pair2<S>::pack(fv[A])), ...);
    }(std::make_integer_sequence<int, Q>{});
  }
}

// Inverse of gather: put canonical pre-collision values fv of cell (x,y,z)
// where the step parity keeps them (checkpoint restore / init).  These two
// helpers serve the kernels off the step path (init, read-back, writes,
// reductions, extrapolation faces) and always index with 64 bits.
template <int Q, typename S, typename R, bool ODD>
__host__ __device__ __forceinline__ void put_canonical(const Domain<R>& d, S* __restrict__ f,
                                                       int x, int y, int z, const R* fv) {
  const int64_t N = d.N;
  const int i = x + d.nx * (y + d.ny * z);
  if constexpr (!ODD) {
    [&]<int... A>(std::integer_sequence<int, A...>) {
      (Codec<S, R>::store(f + A * N + i, fv[A]), ...);
    }(std::make_integer_sequence<int, Q>{});
  } else {
    const Links L = make_links(d, x, y, z);
    [&]<int... A>(std::integer_sequence<int, A...>) {
      (
          [&] {
            int off, mirror;
            bool ghost;
            link_of<Q, A, -1>(L, off, ghost, mirror);
            R v = fv[A];
            const int faces = link_faces<Q, A, -1>(L);
            if (faces)
              v -= R(6.0 * Lattice<Q>::w(A)) *
                   ghost_dot(d, L.edge, faces, Lattice<Q>::c(A, 0), Lattice<Q>::c(A, 1),
                             Lattice<Q>::c(A, 2));
            const int64_t idx =
                ghost ? (A * N + i) : (opposite_mirror_rt<Q, A>(mirror) * N + i + off);
            Codec<S, R>::store(f + idx, v);
          }(),
          ...);
    }(std::make_integer_sequence<int, Q>{});
  }
}

// Canonical pre-collision populations of cell (x,y,z) at any parity.
template <int Q, typename S, typename R, bool ODD>
__host__ __device__ __forceinline__ void get_canonical(const Domain<R>& d, const S* __restrict__ f,
                                                       int x, int y, int z, R* fv) {
  const int i = x + d.nx * (y + d.ny * z);
  if constexpr (!ODD) {
    Links L{};
    gather<Q, S, R, false, false, true, true, true>(d, f, i, L, fv);
  } else {
    gather<Q, S, R, true, false, true, true, true>(d, f, i, make_links(d, x, y, z), fv);
  }
}

}  // namespace lbm
