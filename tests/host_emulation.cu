// Host build of the CUDA step's per-cell code (gather, collide, scatter) for
// CPU tests: cells are updated one after another, which gives the same result
// as the parallel kernel because every cell reads and writes only its own
// set of 2Q slots.  Test infrastructure only.
#include <cstdint>
#include <cmath>

#include "../paper_1503_03337_gb300/csrc/lbm_kernels.cuh"
#include "../paper_1503_03337_gb300/csrc/lbm_neq.cuh"

using namespace lbm;

static int g_sr = 0;
static int g_wide = 0;  // the step's 64-bit-offset (WIDE) instantiations

// fn.template operator()<Q>() for Q = 14, 18 or 26; -1 for any other Q
template <typename Fn>
static int with_q(int Q, Fn&& fn) {
  switch (Q) {
    case 14: fn.template operator()<14>(); return 0;
    case 18: fn.template operator()<18>(); return 0;
    case 26: fn.template operator()<26>(); return 0;
  }
  return -1;
}
static const uint32_t* g_solid = nullptr;  // solid-link words (Domain::solid) or null

template <int Q, typename S, typename R>
static void step_typed(void* f, int nx, int ny, int nz, const int* per, int moving, int sym, const int* eaxis, const double* escale,
                       const double* uw, const double* s, const double* F, int64_t n) {
  Domain<R> d{};
  d.f = f;
  d.nx = nx; d.ny = ny; d.nz = nz;
  d.N = (int64_t)nx * ny * nz;
  d.moving = moving;
  d.sym = sym;
  d.solid = g_solid;
  for (int face = 0; face < 6; ++face) {
    d.edge_axis[face] = eaxis ? eaxis[face] : 0;
    d.edge_scale[face][0] = R(escale ? escale[2 * face] : 1.0);
    d.edge_scale[face][1] = R(escale ? escale[2 * face + 1] : 1.0);
  }
  for (int k = 0; k < 3; ++k) d.per[k] = per[k];
  for (int face = 0; face < 6; ++face)
    for (int k = 0; k < 3; ++k) d.uw[face][k] = R(uw[3 * face + k]);
  d.s.sc = R(s[0]); d.s.se = R(s[1]); d.s.sq = R(s[2]);
  d.s.snu = R(s[3]); d.s.spi = R(s[4]); d.s.st = R(s[5]);
  scale_rows<Q>(d.s);
  for (int k = 0; k < 3; ++k) d.F[k] = R(F[k]);
  d.key = mix32(0x5eedu ^ uint32_t(n) * 0x632be5abu);
  fill_offsets<Q>(d);
  const bool force = F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0;
  // one cell of the step kernel: parity, force and rounding as launched
  auto cell = [&]<bool WIDE>(int x, int y, int z, int xl, int xh) {
    S* fs = static_cast<S*>(f);
    if constexpr (Stochastic<S>::enabled) {
      if (g_sr) {
        if (n & 1) update_cell<Q, S, R, true, true, true, false, WIDE>(d, fs, x, y, z, xl, xh);
        else update_cell<Q, S, R, false, true, true, false, WIDE>(d, fs, x, y, z, xl, xh);
        return;
      }
    }
    if (n & 1) {
      if (force) update_cell<Q, S, R, true, true, false, false, WIDE>(d, fs, x, y, z, xl, xh);
      else update_cell<Q, S, R, true, false, false, false, WIDE>(d, fs, x, y, z, xl, xh);
    } else {
      if (force) update_cell<Q, S, R, false, true, false, false, WIDE>(d, fs, x, y, z, xl, xh);
      else update_cell<Q, S, R, false, false, false, false, WIDE>(d, fs, x, y, z, xl, xh);
    }
  };
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        // the 32-wide x-range a warp of a 32-multiple-wide block would cover
        const int xl = x & ~31, xh = xl + 31;
        if (g_wide) cell.template operator()<true>(x, y, z, xl, xh);
        else cell.template operator()<false>(x, y, z, xl, xh);
      }
}

template <int Q, typename S, typename R, bool ODD>
static void canonical_typed(void* f, int nx, int ny, int nz, const int* per, int moving, int sym, const int* eaxis, const double* escale,
                            const double* uw, double* out, int to_storage) {
  Domain<R> d{};
  d.f = f;
  d.nx = nx; d.ny = ny; d.nz = nz;
  d.N = (int64_t)nx * ny * nz;
  fill_offsets<Q>(d);
  d.moving = moving;
  d.sym = sym;
  d.solid = g_solid;
  for (int face = 0; face < 6; ++face) {
    d.edge_axis[face] = eaxis ? eaxis[face] : 0;
    d.edge_scale[face][0] = R(escale ? escale[2 * face] : 1.0);
    d.edge_scale[face][1] = R(escale ? escale[2 * face + 1] : 1.0);
  }
  for (int k = 0; k < 3; ++k) d.per[k] = per[k];
  for (int face = 0; face < 6; ++face)
    for (int k = 0; k < 3; ++k) d.uw[face][k] = R(uw[3 * face + k]);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int64_t i = x + (int64_t)nx * (y + (int64_t)ny * z);
        R fv[Q];
        if (to_storage) {
          for (int a = 0; a < Q; ++a) fv[a] = R(out[a * d.N + i]);
          put_canonical<Q, S, R, ODD>(d, static_cast<S*>(f), x, y, z, fv);
        } else {
          get_canonical<Q, S, R, ODD>(d, static_cast<const S*>(f), x, y, z, fv);
          for (int a = 0; a < Q; ++a) out[a * d.N + i] = double(fv[a]);
        }
      }
}

template <typename S, typename R>
static int canon_any(int Q, void* f, int nx, int ny, int nz, const int* per, int moving, int sym, const int* eaxis, const double* escale,
                     const double* uw, double* canon, int64_t n, int to_storage) {
  const bool odd = n & 1;
  return with_q(Q, [&]<int QQ>() {
    if (odd) canonical_typed<QQ, S, R, true>(f, nx, ny, nz, per, moving, sym, eaxis, escale, uw, canon, to_storage);
    else canonical_typed<QQ, S, R, false>(f, nx, ny, nz, per, moving, sym, eaxis, escale, uw, canon, to_storage);
  });
}

// The extrapolation pass over every boundary node, on the populations of
// step n (FP64 storage): uw holds the velocity of every velocity face, pb the
// pressure of every pressure face at time level n, F the force at n.
template <int Q, bool ODD>
static void neq_typed(void* f, int nx, int ny, int nz, const int* per, int moving, int sym,
                      const double* uw, int vel, int pre, const double* pb, const double* F) {
  Domain<double> d{};
  d.f = f;
  d.nx = nx; d.ny = ny; d.nz = nz;
  d.N = (int64_t)nx * ny * nz;
  d.moving = moving;
  d.sym = sym;
  for (int k = 0; k < 3; ++k) d.per[k] = per[k];
  for (int face = 0; face < 6; ++face) {
    d.edge_axis[face] = 0;
    d.edge_scale[face][0] = d.edge_scale[face][1] = 1.0;
    for (int k = 0; k < 3; ++k) d.uw[face][k] = uw[3 * face + k];
  }
  for (int k = 0; k < 3; ++k) d.F[k] = F[k];
  fill_offsets<Q>(d);
  NeqArgs a{};
  a.vel = vel;
  a.pre = pre;
  const int plane[3] = {ny * nz, nx * nz, nx * ny};
  for (int face = 0; face < 6; ++face) {
    a.off[face + 1] = a.off[face] + ((((vel | pre) >> face) & 1) ? plane[face >> 1] : 0);
    a.pb[face] = pb[face];
  }
  for (int t = 0; t < a.off[6]; ++t) neq_node<Q, double, double, ODD>(d, a, t);
}

extern "C" {
void emu_set_stochastic(int on) { g_sr = on; }
void emu_set_wide(int on) { g_wide = on; }

// Solid-link words of a byte mask (the device builder's per-cell code).
int emu_solid_links(int Q, int nx, int ny, int nz, int per, int sym, const uint8_t* bytes,
                    uint32_t* out) {
  const int64_t N = (int64_t)nx * ny * nz;
  return with_q(Q, [&]<int QQ>() {
    for (int64_t i = 0; i < N; ++i) out[i] = solid_link_bits<QQ>(nx, ny, nz, per, sym, bytes, i);
  });
}
void emu_set_solid(const uint32_t* links) { g_solid = links; }

int emu_neq(int Q, void* f, int nx, int ny, int nz, const int* per, int moving, int sym,
            const double* uw, int vel, int pre, const double* pb, const double* F, int64_t n) {
  const bool odd = n & 1;
  return with_q(Q, [&]<int QQ>() {
    if (odd) neq_typed<QQ, true>(f, nx, ny, nz, per, moving, sym, uw, vel, pre, pb, F);
    else neq_typed<QQ, false>(f, nx, ny, nz, per, moving, sym, uw, vel, pre, pb, F);
  });
}

// storage: 0 double, 1 float, 2 half, 3 bfloat16
int emu_step(int Q, int storage, void* f, int nx, int ny, int nz, const int* per, int moving, int sym, const int* eaxis, const double* escale,
             const double* uw, const double* s, const double* F, int64_t n) {
  if (storage < 0 || storage > 3) return -1;
  return with_q(Q, [&]<int QQ>() {
    if (storage == 0) step_typed<QQ, double, double>(f, nx, ny, nz, per, moving, sym, eaxis, escale, uw, s, F, n);
    else if (storage == 1) step_typed<QQ, float, float>(f, nx, ny, nz, per, moving, sym, eaxis, escale, uw, s, F, n);
    else if (storage == 2) step_typed<QQ, __half, float>(f, nx, ny, nz, per, moving, sym, eaxis, escale, uw, s, F, n);
    else step_typed<QQ, __nv_bfloat16, float>(f, nx, ny, nz, per, moving, sym, eaxis, escale, uw, s, F, n);
  });
}

// canonical f (FP64) <-> storage layout of parity n (double storage only)
int emu_canonical_storage(int Q, int storage, void* f, int nx, int ny, int nz, const int* per,
                          int moving, int sym, const int* eaxis, const double* escale, const double* uw, double* canon, int64_t n,
                          int to_storage) {
  switch (storage) {
    case 0: return canon_any<double, double>(Q, f, nx, ny, nz, per, moving, sym, eaxis, escale, uw, canon, n, to_storage);
    case 1: return canon_any<float, float>(Q, f, nx, ny, nz, per, moving, sym, eaxis, escale, uw, canon, n, to_storage);
    case 2: return canon_any<__half, float>(Q, f, nx, ny, nz, per, moving, sym, eaxis, escale, uw, canon, n, to_storage);
    case 3: return canon_any<__nv_bfloat16, float>(Q, f, nx, ny, nz, per, moving, sym, eaxis, escale, uw, canon, n, to_storage);
  }
  return -1;
}

int emu_canonical(int Q, void* f, int nx, int ny, int nz, const int* per, int moving, int sym, const int* eaxis, const double* escale,
                  const double* uw, double* canon, int64_t n, int to_storage) {
  return canon_any<double, double>(Q, f, nx, ny, nz, per, moving, sym, eaxis, escale, uw, canon, n,
                                   to_storage);
}

int emu_collide(int Q, const double* s, double* f, const double* F) {
  Rates<double> r{s[0], s[1], s[2], s[3], s[4], s[5], {}, {}, {}};
  double ux, uy, uz;
  return with_q(Q, [&]<int QQ>() {
    scale_rows<QQ>(r);
    collide<QQ, true>(f, r, F[0], F[1], F[2], ux, uy, uz);
  });
}
}
