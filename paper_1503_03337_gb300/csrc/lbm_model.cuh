// Lattice tables, moment basis, rates, storage codecs and arithmetic
// helpers of the iD3Q14 (Sec. 3) and iD3Q18 (App. B) incompressible models,
// and of the iD3Q26 model that the same construction gives on the D3Q27 set
// without c_0 (App. B's closing remark).
//
// Everything that depends only on the lattice is a constexpr function: the
// rows of T are the orthogonal basis vectors phi_k of Sec. 3 (Eq. m, after
// orthogonalisation) and App. B (Eq. appendix_m18), evaluated on the
// velocity set, and no matrix is stored anywhere.  The transform itself is
// in lbm_factored.cuh, checked against phi at compile time, and the
// collision in lbm_collide.cuh.
//
// Every direction a has an opposite abar (Q is even and there is no rest
// direction), and every row of T is either even (T_k,abar = T_k,a: P, e and
// the second-order moments) or odd (T_k,abar = -T_k,a: j, q, t).  The
// transform therefore runs on pair sums s = f_a + f_abar (even rows) and
// pair differences d = f_a - f_abar (odd rows), which halves its cost.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <utility>

namespace lbm {

// ---------------------------------------------------------------------------
// Velocity sets and weights
// ---------------------------------------------------------------------------
template <int Q>
struct Lattice;

// iD3Q14, Sec. 3: c_1..c_6 on the axes, c_7..c_14 on the cube diagonals.
template <>
struct Lattice<14> {
  static constexpr int Q = 14;
  __host__ __device__ static constexpr int c(int a, int d) {
    const int v[14][3] = {{1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
                          {0, 0, 1},   {0, 0, -1},  {1, 1, 1},   {-1, 1, 1},
                          {1, -1, 1},  {-1, -1, 1}, {1, 1, -1},  {-1, 1, -1},
                          {1, -1, -1}, {-1, -1, -1}};
    return v[a][d];
  }
  // D3Q15 weights of the discarded rest direction and of the stored ones
  // (the only weights for which Eq. meq equals T f_eq).
  static constexpr double w0 = 2.0 / 9.0;
  __host__ __device__ static constexpr double w(int a) {
    return a < 6 ? 1.0 / 9.0 : 1.0 / 72.0;
  }
};

// iD3Q18, App. B: c_1..c_6 on the axes, c_7..c_18 on the face diagonals.
template <>
struct Lattice<18> {
  static constexpr int Q = 18;
  __host__ __device__ static constexpr int c(int a, int d) {
    const int v[18][3] = {{1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                          {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, 1, 0},
                          {1, -1, 0}, {-1, -1, 0}, {1, 0, 1},  {-1, 0, 1},
                          {1, 0, -1}, {-1, 0, -1}, {0, 1, 1},  {0, -1, 1},
                          {0, 1, -1}, {0, -1, -1}};
    return v[a][d];
  }
  static constexpr double w0 = 1.0 / 3.0;
  __host__ __device__ static constexpr double w(int a) {
    return a < 6 ? 1.0 / 18.0 : 1.0 / 36.0;
  }
};

// iD3Q26: the 26 velocities of D3Q27 without c_0 -- the axes and face
// diagonals in the order of iD3Q18, then the cube diagonals in the order of
// iD3Q14 -- with the D3Q27 weights (8/27 for the discarded rest direction,
// 2/27, 1/54 and 1/216 for the three shells).
template <>
struct Lattice<26> {
  static constexpr int Q = 26;
  __host__ __device__ static constexpr int c(int a, int d) {
    return a < 18 ? Lattice<18>::c(a, d) : Lattice<14>::c(a - 12, d);
  }
  static constexpr double w0 = 8.0 / 27.0;
  __host__ __device__ static constexpr double w(int a) {
    return a < 6 ? 2.0 / 27.0 : (a < 18 ? 1.0 / 54.0 : 1.0 / 216.0);
  }
};

template <int Q>
__host__ __device__ constexpr int opposite(int a) {
  for (int b = 0; b < Q; ++b)
    if (Lattice<Q>::c(b, 0) == -Lattice<Q>::c(a, 0) &&
        Lattice<Q>::c(b, 1) == -Lattice<Q>::c(a, 1) &&
        Lattice<Q>::c(b, 2) == -Lattice<Q>::c(a, 2))
      return b;
  return -1;
}

// i-th pair representative: the i-th direction (in index order) whose
// opposite has a larger index.
template <int Q>
__host__ __device__ constexpr int pair_rep(int i) {
  int seen = 0;
  for (int a = 0; a < Q; ++a)
    if (opposite<Q>(a) > a) {
      if (seen == i) return a;
      ++seen;
    }
  return -1;
}

// ---------------------------------------------------------------------------
// Moment basis
// ---------------------------------------------------------------------------
enum RowKind { ROW_P, ROW_E, ROW_J, ROW_Q, ROW_NU, ROW_PI, ROW_T };

template <int Q>
__host__ __device__ constexpr int phi(int k, int a) {
  const int cx = Lattice<Q>::c(a, 0), cy = Lattice<Q>::c(a, 1),
            cz = Lattice<Q>::c(a, 2);
  const int n2 = cx * cx + cy * cy + cz * cz;
  if (Q == 14) {
    // P, e, jx, qx, jy, qy, jz, qz, 3pxx, pww, pxy, pyz, pxz, txyz
    switch (k) {
      case 0: return 1;
      case 1: return (7 * n2 - 15) / 2;
      case 2: return cx;
      case 3: return (5 * n2 - 13) * cx / 2;
      case 4: return cy;
      case 5: return (5 * n2 - 13) * cy / 2;
      case 6: return cz;
      case 7: return (5 * n2 - 13) * cz / 2;
      case 8: return 3 * cx * cx - n2;
      case 9: return cy * cy - cz * cz;
      case 10: return cx * cy;
      case 11: return cy * cz;
      case 12: return cx * cz;
      case 13: return cx * cy * cz;
    }
  } else if (Q == 26) {
    // The monomials 1, |c|^2, c_x, |c|^2 c_x, ..., 3c_x^2 - |c|^2,
    // |c|^2 (3c_x^2 - |c|^2), c_y^2 - c_z^2, |c|^2 (c_y^2 - c_z^2), c_x c_y,
    // c_y c_z, c_x c_z, the three t's, |c|^4, |c|^4 c_x, |c|^4 c_y, |c|^4 c_z,
    // |c|^2 c_x c_y, |c|^2 c_y c_z, |c|^2 c_x c_z and c_x c_y c_z, each
    // orthogonalised against the ones before it (Sec. 3's recipe) and scaled
    // to integers.  On this set a function of |c|^2 is a function of the
    // shell (sizes 6, 12, 8), so orthogonalising a monomial g(|c|^2) h(c)
    // against the lower ones only changes g, to the quadratic in |c|^2 whose
    // shell values make it orthogonal with the shell weights of h^2:
    //   |c|^2       -> 13|c|^2 - 27                     (-14, -1, 12)
    //   |c|^2 c_x   -> (3|c|^2 - 7) c_x                 (-4, -1, 2)
    //   |c|^2 (3c_x^2 - |c|^2) -> (3|c|^2 - 5)(...)     (-2, 1, -)
    //   |c|^4       -> (15|c|^4 - 61|c|^2 + 54) / 2     (4, -4, 3)
    //   |c|^4 c_x   -> (9|c|^4 - 39|c|^2 + 38) / 2 c_x  (4, -2, 1)
    //   |c|^2 c_x c_y -> (3|c|^2 - 8) c_x c_y           (-, -2, 1)
    // The remaining monomials are already orthogonal to the ones before them
    // (by their parity in each of c_x, c_y, c_z and their cubic symmetry);
    // basis_ok checks all of it at compile time.  The |c|^6 and
    // c_x^2 c_y^2 c_z^2 monomials are left out: (1 - c_x^2)(1 - c_y^2)(1 -
    // c_z^2) = 0 on these velocities makes them dependent on the others.
    switch (k) {
      case 0: return 1;
      case 1: return 13 * n2 - 27;
      case 2: return cx;
      case 3: return (3 * n2 - 7) * cx;
      case 4: return cy;
      case 5: return (3 * n2 - 7) * cy;
      case 6: return cz;
      case 7: return (3 * n2 - 7) * cz;
      case 8: return 3 * cx * cx - n2;
      case 9: return (3 * n2 - 5) * (3 * cx * cx - n2);
      case 10: return cy * cy - cz * cz;
      case 11: return (3 * n2 - 5) * (cy * cy - cz * cz);
      case 12: return cx * cy;
      case 13: return cy * cz;
      case 14: return cx * cz;
      case 15: return (cy * cy - cz * cz) * cx;
      case 16: return (cz * cz - cx * cx) * cy;
      case 17: return (cx * cx - cy * cy) * cz;
      case 18: return (15 * n2 * n2 - 61 * n2 + 54) / 2;
      case 19: return (9 * n2 * n2 - 39 * n2 + 38) / 2 * cx;
      case 20: return (9 * n2 * n2 - 39 * n2 + 38) / 2 * cy;
      case 21: return (9 * n2 * n2 - 39 * n2 + 38) / 2 * cz;
      case 22: return (3 * n2 - 8) * cx * cy;
      case 23: return (3 * n2 - 8) * cy * cz;
      case 24: return (3 * n2 - 8) * cx * cz;
      case 25: return cx * cy * cz;
    }
  } else {
    // P, e, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz,
    // tx, ty, tz
    switch (k) {
      case 0: return 1;
      case 1: return 3 * n2 - 5;
      case 2: return cx;
      case 3: return (5 * n2 - 9) * cx;
      case 4: return cy;
      case 5: return (5 * n2 - 9) * cy;
      case 6: return cz;
      case 7: return (5 * n2 - 9) * cz;
      case 8: return 3 * cx * cx - n2;
      case 9: return (3 * n2 - 5) * (3 * cx * cx - n2);
      case 10: return cy * cy - cz * cz;
      case 11: return (3 * n2 - 5) * (cy * cy - cz * cz);
      case 12: return cx * cy;
      case 13: return cy * cz;
      case 14: return cx * cz;
      case 15: return (cy * cy - cz * cz) * cx;
      case 16: return (cz * cz - cx * cx) * cy;
      case 17: return (cx * cx - cy * cy) * cz;
    }
  }
  return 0;
}

// Row k is even if T_k,abar = T_k,a for every direction (else odd).
template <int Q>
__host__ __device__ constexpr bool row_even(int k) {
  for (int a = 0; a < Q; ++a)
    if (phi<Q>(k, a) != phi<Q>(k, opposite<Q>(a))) return false;
  return true;
}

template <int Q>
__host__ __device__ constexpr int row_norm(int k) {
  int s = 0;
  for (int a = 0; a < Q; ++a) s += phi<Q>(k, a) * phi<Q>(k, a);
  return s;
}

// Compile-time checks of the basis: every row has a definite parity under
// c -> -c, rows are mutually orthogonal (so T^-1 = T' D^-1), and the
// conserved rows are P = sum f and j = sum c f.
template <int Q>
__host__ __device__ constexpr bool basis_ok() {
  for (int a = 0; a < Q; ++a)
    if (opposite<Q>(a) < 0 || opposite<Q>(opposite<Q>(a)) != a) return false;
  for (int k = 0; k < Q; ++k) {
    const bool even = row_even<Q>(k);
    for (int a = 0; a < Q; ++a) {
      const int t = phi<Q>(k, a), tb = phi<Q>(k, opposite<Q>(a));
      if (even ? (t != tb) : (t != -tb)) return false;
    }
    for (int l = 0; l < k; ++l) {
      int dot = 0;
      for (int a = 0; a < Q; ++a) dot += phi<Q>(k, a) * phi<Q>(l, a);
      if (dot != 0) return false;
    }
    if (row_norm<Q>(k) <= 0) return false;
  }
  for (int a = 0; a < Q; ++a)
    if (phi<Q>(0, a) != 1 || phi<Q>(2, a) != Lattice<Q>::c(a, 0) ||
        phi<Q>(4, a) != Lattice<Q>::c(a, 1) || phi<Q>(6, a) != Lattice<Q>::c(a, 2))
      return false;
  return true;
}
static_assert(basis_ok<14>(), "iD3Q14 moment basis is inconsistent");
static_assert(basis_ok<18>(), "iD3Q18 moment basis is inconsistent");
static_assert(basis_ok<26>(), "iD3Q26 moment basis is inconsistent");

// ---------------------------------------------------------------------------
// Storage codec: populations live in S, arithmetic runs in R.
// ---------------------------------------------------------------------------
template <typename S, typename R>
struct Codec;
// load_cg reads through L2 only (ld.global.cg).  A kernel that runs several
// steps in one launch must read populations this way: L1 is not coherent
// between SMs, and a line cached in one step could be stale in the next.
template <typename R>
struct Codec<double, R> {
  __host__ __device__ static R value(double v) { return R(v); }
  __host__ __device__ static R load(const double* p) {
#ifdef __CUDA_ARCH__
    return R(__ldg(p));
#else
    return R(*p);
#endif
  }
  __host__ __device__ static R load_cg(const double* p) {
#ifdef __CUDA_ARCH__
    return R(__ldcg(p));
#else
    return R(*p);
#endif
  }
  __host__ __device__ static void store(double* p, R v) { *p = double(v); }
};
template <typename R>
struct Codec<float, R> {
  __host__ __device__ static R value(float v) { return R(v); }
  __host__ __device__ static R load(const float* p) { return R(*p); }
  __host__ __device__ static R load_cg(const float* p) {
#ifdef __CUDA_ARCH__
    return R(__ldcg(p));
#else
    return R(*p);
#endif
  }
  __host__ __device__ static void store(float* p, R v) { *p = float(v); }
};
template <typename R>
struct Codec<__half, R> {
  __host__ __device__ static R value(__half v) { return R(__half2float(v)); }
  __host__ __device__ static R load(const __half* p) { return R(__half2float(*p)); }
  __host__ __device__ static R load_cg(const __half* p) {
#ifdef __CUDA_ARCH__
    return R(__half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short*>(p)))));
#else
    return R(__half2float(*p));
#endif
  }
  __host__ __device__ static void store(__half* p, R v) { *p = __float2half_rn(float(v)); }
};
template <typename R>
struct Codec<__nv_bfloat16, R> {
  __host__ __device__ static R value(__nv_bfloat16 v) { return R(__bfloat162float(v)); }
  __host__ __device__ static R load(const __nv_bfloat16* p) {
    return R(__bfloat162float(*p));
  }
  __host__ __device__ static R load_cg(const __nv_bfloat16* p) {
#ifdef __CUDA_ARCH__
    return R(__bfloat162float(
        __ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short*>(p)))));
#else
    return R(__bfloat162float(*p));
#endif
  }
  __host__ __device__ static void store(__nv_bfloat16* p, R v) {
    *p = __float2bfloat16_rn(float(v));
  }
};

template <typename S, typename R, bool CG>
__host__ __device__ __forceinline__ R load_pop(const S* p) {
  if constexpr (CG) return Codec<S, R>::load_cg(p);
  else return Codec<S, R>::load(p);
}

// ---------------------------------------------------------------------------
// Stochastic rounding for 16-bit storage.  Rounding to nearest loses every
// per-step change smaller than half a storage ulp in the same direction
// (stagnation), which biases slowly varying populations.  Rounding up with
// probability equal to the discarded fraction makes every store unbiased.
// The random bits come from a counter-based hash of (cell, direction, step),
// so runs are reproducible and independent of launch shape or batching.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
  // integer finaliser (xorshift-multiply, constants from public hash designs)
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
__host__ __device__ __forceinline__ uint32_t mix32_short(uint32_t x) {
  x ^= x >> 15;
  x *= 0x2c1b3c6du;
  x ^= x >> 12;
  return x;
}

__host__ __device__ __forceinline__ uint32_t f32_bits(float v) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(v);
#else
  uint32_t b;
  memcpy(&b, &v, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ float bits_f32(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float v;
  memcpy(&v, &b, 4);
  return v;
#endif
}

// Stochastic rounding of two FP32 values into one 32-bit word of two 16-bit
// values, hi <- a and lo <- b, from 32 random bits r.  Each value becomes one
// of its two 16-bit neighbours with probability proportional to its distance
// to the other, so the stored value is unbiased:
//   FP16: |v| / s + k / 8192 rounded down, times s, with s the FP16 spacing
//         at |v| (2^-24 below 2^-14) and k = r[28:16] (hi) or r[12:0] (lo);
//   BF16: the 16 random bits r[31:16] (hi) or r[15:0] (lo) added to the
//         16 bits of the FP32 magnitude that BF16 drops, then truncated.
// On the device each pair is one conversion instruction (cvt.rs.f16x2 /
// .bf16x2 of sm_100 and later, whose bit layout and rounding are exactly
// these); host builds compute the same bits.  Finite inputs below the
// format's largest value.
template <typename S>
struct Stochastic {
  static constexpr bool enabled = false;
};
template <>
struct Stochastic<__half> {
  static constexpr bool enabled = true;
  __host__ static float round_host(float v, uint32_t k) {
    const uint32_t b = f32_bits(v), mag = b & 0x7fffffffu, sign = b & 0x80000000u;
    if (mag >= 0x7f800000u) return v;
    if (mag >= 0x38800000u)  // |v| >= 2^-14: drop 13 of the 23 mantissa bits
      return bits_f32(sign | ((mag + k) & ~0x1fffu));
    // subnormal FP16 spacing 2^-24: count spacings, exactly in double
    const double q = std::floor(double(bits_f32(mag)) * 16777216.0 + double(k) / 8192.0);
    return bits_f32(sign | f32_bits(float(q / 16777216.0)));
  }
  __host__ __device__ static uint32_t pack2(float a, float b, uint32_t r) {
#ifdef __CUDA_ARCH__
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(r));
    return d;
#else
    const __half ha = __float2half_rz(round_host(a, (r >> 16) & 0x1fffu));
    const __half hb = __float2half_rz(round_host(b, r & 0x1fffu));
    uint16_t ua, ub;
    memcpy(&ua, &ha, 2);
    memcpy(&ub, &hb, 2);
    return (uint32_t(ua) << 16) | ub;
#endif
  }
};
template <>
struct Stochastic<__nv_bfloat16> {
  static constexpr bool enabled = true;
  __host__ static uint16_t round_host(float v, uint32_t k) {
    const uint32_t b = f32_bits(v), mag = b & 0x7fffffffu;
    if (mag >= 0x7f800000u) return uint16_t(b >> 16);
    return uint16_t(((b & 0x80000000u) | ((mag + k) & ~0xffffu)) >> 16);
  }
  __host__ __device__ static uint32_t pack2(float a, float b, uint32_t r) {
#ifdef __CUDA_ARCH__
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(r));
    return d;
#else
    return (uint32_t(round_host(a, r >> 16)) << 16) | round_host(b, r & 0xffffu);
#endif
  }
};

// ---------------------------------------------------------------------------
// Two adjacent cells at once (2-byte storage): a packed pair of FP32
// values.  On the device every add, multiply and multiply-add is one packed
// FP32x2 instruction (__fadd2_rn / __fmul2_rn / __ffma2_rn of sm_100 and
// later), so the collision of two cells issues the instructions of one.
// Arithmetic stays IEEE FP32, rounded to nearest, per component.
// ---------------------------------------------------------------------------
// (The scalar branches serve host builds of this header; device code is
// only ever built for sm_103a.)
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
#define LBM_PACKED_F32X2 1
#else
#define LBM_PACKED_F32X2 0
#endif

struct pf2 {
  float2 v;
  pf2() = default;
  __host__ __device__ pf2(float s) : v(make_float2(s, s)) {}  // broadcast
  __host__ __device__ pf2(float a, float b) : v(make_float2(a, b)) {}
};

__host__ __device__ __forceinline__ pf2 pf2_from(float2 v) {
  pf2 r;
  r.v = v;
  return r;
}
__host__ __device__ __forceinline__ pf2 operator+(pf2 a, pf2 b) {
#if LBM_PACKED_F32X2
  return pf2_from(__fadd2_rn(a.v, b.v));
#else
  return pf2(a.v.x + b.v.x, a.v.y + b.v.y);
#endif
}
__host__ __device__ __forceinline__ pf2 operator*(pf2 a, pf2 b) {
#if LBM_PACKED_F32X2
  return pf2_from(__fmul2_rn(a.v, b.v));
#else
  return pf2(a.v.x * b.v.x, a.v.y * b.v.y);
#endif
}
// a * b + c
__host__ __device__ __forceinline__ pf2 fmadd(pf2 a, pf2 b, pf2 c) {
#if LBM_PACKED_F32X2
  return pf2_from(__ffma2_rn(a.v, b.v, c.v));
#else
  return pf2(std::fma(a.v.x, b.v.x, c.v.x), std::fma(a.v.y, b.v.y, c.v.y));
#endif
}
__host__ __device__ __forceinline__ pf2 operator-(pf2 a, pf2 b) {
  return fmadd(b, pf2(-1.0f), a);
}
__host__ __device__ __forceinline__ pf2 operator-(pf2 a) { return a * pf2(-1.0f); }
__host__ __device__ __forceinline__ pf2 operator*(float s, pf2 a) { return pf2(s) * a; }
__host__ __device__ __forceinline__ pf2 operator*(pf2 a, float s) { return a * pf2(s); }
__host__ __device__ __forceinline__ pf2 operator+(pf2 a, float s) { return a + pf2(s); }
__host__ __device__ __forceinline__ pf2 operator-(pf2 a, float s) { return a - pf2(s); }
__host__ __device__ __forceinline__ pf2& operator+=(pf2& a, pf2 b) { return a = a + b; }
__host__ __device__ __forceinline__ pf2& operator-=(pf2& a, pf2 b) { return a = a - b; }

__host__ __device__ __forceinline__ float fmadd(float a, float b, float c) { return a * b + c; }
__host__ __device__ __forceinline__ double fmadd(double a, double b, double c) {
  return a * b + c;
}
// integer form, for compile-time checks of the transforms
__host__ __device__ constexpr int fmadd(int a, int b, int c) { return a * b + c; }

// acc + C x (term_add) and C x (term_first) for a compile-time integer C: an
// add or subtract for C = +-1, else one multiply(-add).
template <int C, typename V>
__host__ __device__ __forceinline__ constexpr V term_first(V x) {
  if constexpr (C == 1) return x;
  else if constexpr (C == -1) return -x;
  else return V(C) * x;
}
template <int C, typename V>
__host__ __device__ __forceinline__ constexpr V term_add(V acc, V x) {
  if constexpr (C == 1) return acc + x;
  else if constexpr (C == -1) return acc - x;
  else return fmadd(V(C), x, acc);
}

template <typename R>
struct Rates {
  R sc, se, sq, snu, spi, st;
  // Per row K of T, with D_K its norm: k[K] = s_K / D_K,
  // h[K] = (1 - s_K/2) / D_K (for the momentum rows, which carry only the
  // force, h[K] = 1 / D_K) and g[K] = (1 - s_K) / D_K, so that the
  // post-collision row over its norm is g m + k m_eq + h S_F.  Filled once
  // per launch by scale_rows, so the collision multiplies each row once.
  R k[26], h[26], g[26];
};

// Relaxation rate of row K (Eq. sD3Q15meaning / Eq. sD3Q19): conserved rows
// s_c, energy s_e, heat flux s_q, the stress rows s_nu (the pi rows of Q18
// s_pi), the third-order rows s_t.  The paper gives no rates for iD3Q26;
// its rows take the rate of the iD3Q18 row they extend: |c|^4 that of e,
// the |c|^4 c rows that of q, the |c|^2 c_x c_y rows that of pi, and
// c_x c_y c_z that of t.
template <int Q, typename R>
__host__ __device__ constexpr R rate_of(const Rates<R>& r, int K) {
  if (K == 0 || K == 2 || K == 4 || K == 6) return r.sc;
  if (K == 1) return r.se;
  if (K == 3 || K == 5 || K == 7) return r.sq;
  if (Q == 14) return K == 13 ? r.st : r.snu;
  if (K == 9 || K == 11) return r.spi;
  if (Q == 26 && K >= 18) {
    if (K == 18) return r.se;
    if (K <= 21) return r.sq;
    return K == 25 ? r.st : r.spi;
  }
  return K >= 15 ? r.st : r.snu;
}

template <int Q, typename R>
__host__ __device__ inline void scale_rows(Rates<R>& r) {
  for (int K = 0; K < 26; ++K) {
    r.k[K] = R(0);
    r.h[K] = R(0);
    r.g[K] = R(0);
  }
  for (int K = 0; K < Q; ++K) {
    const R inv = R(1.0 / row_norm<Q>(K));
    const R sk = rate_of<Q>(r, K);
    r.k[K] = sk * inv;
    r.h[K] = (K == 2 || K == 4 || K == 6) ? inv : (R(1) - R(0.5) * sk) * inv;
    r.g[K] = (R(1) - sk) * inv;
  }
}

// ---------------------------------------------------------------------------
// Equilibrium moments from their definition m_eq = T f_eq (Eq. mrteqvT), for
// a model without printed closed forms (iD3Q26).  With
//   f_eq,a = w_a [3p + 3 c_a.u + 9/2 (c_a.u)^2 - 3/2 u^2]
// (the incompressible equilibrium, Eq. edf, c_s^2 = 1/3), row K is
//   m_eq,K = A_K (3p - 3/2 u^2) + 3 sum_d B_Kd u_d + 9/2 sum_de C_Kde u_d u_e
// with the compile-time weighted sums A_K = sum_a phi_K w_a,
// B_Kd = sum_a phi_K w_a c_d and C_Kde = sum_a phi_K w_a c_d c_e.  The Guo
// source (the projection of w_a [3 c.F + 9 (c.u)(c.F) - 3 u.F]) is the
// derivative of the same form along F at fixed p:
//   S_F,K = -3 A_K u.F + 3 sum_d B_Kd F_d + 9 sum_de C_Kde u_d F_e.
// ---------------------------------------------------------------------------
template <int Q>
__host__ __device__ constexpr double eq_a(int K) {
  double s = 0.0;
  for (int a = 0; a < Q; ++a) s += phi<Q>(K, a) * Lattice<Q>::w(a);
  return s;
}
template <int Q>
__host__ __device__ constexpr double eq_b(int K, int d) {
  double s = 0.0;
  for (int a = 0; a < Q; ++a) s += phi<Q>(K, a) * Lattice<Q>::w(a) * Lattice<Q>::c(a, d);
  return s;
}
template <int Q>
__host__ __device__ constexpr double eq_c(int K, int d, int e) {
  double s = 0.0;
  for (int a = 0; a < Q; ++a)
    s += phi<Q>(K, a) * Lattice<Q>::w(a) * Lattice<Q>::c(a, d) * Lattice<Q>::c(a, e);
  return s;
}

// acc + C * x, with C a compile-time constant (no instruction when C = 0)
template <typename V, typename R>
__host__ __device__ __forceinline__ V add_scaled(V acc, double C, V x) {
  return C == 0.0 ? acc : fmadd(V(R(C)), x, acc);
}

// m_eq,K (q3 = 3p - 3/2 u^2; uu = u_x^2, u_y^2, u_z^2, u_x u_y, u_y u_z,
// u_x u_z)
template <int Q, int K, typename V, typename R>
__host__ __device__ __forceinline__ V moment_eq(V q3, V ux, V uy, V uz, const V* uu) {
  constexpr double A = eq_a<Q>(K);
  constexpr double Bx = 3.0 * eq_b<Q>(K, 0), By = 3.0 * eq_b<Q>(K, 1), Bz = 3.0 * eq_b<Q>(K, 2);
  constexpr double Cxx = 4.5 * eq_c<Q>(K, 0, 0), Cyy = 4.5 * eq_c<Q>(K, 1, 1),
                   Czz = 4.5 * eq_c<Q>(K, 2, 2), Cxy = 9.0 * eq_c<Q>(K, 0, 1),
                   Cyz = 9.0 * eq_c<Q>(K, 1, 2), Cxz = 9.0 * eq_c<Q>(K, 0, 2);
  V acc = V(R(0));
  acc = add_scaled<V, R>(acc, A, q3);
  acc = add_scaled<V, R>(acc, Bx, ux);
  acc = add_scaled<V, R>(acc, By, uy);
  acc = add_scaled<V, R>(acc, Bz, uz);
  acc = add_scaled<V, R>(acc, Cxx, uu[0]);
  acc = add_scaled<V, R>(acc, Cyy, uu[1]);
  acc = add_scaled<V, R>(acc, Czz, uu[2]);
  acc = add_scaled<V, R>(acc, Cxy, uu[3]);
  acc = add_scaled<V, R>(acc, Cyz, uu[4]);
  acc = add_scaled<V, R>(acc, Cxz, uu[5]);
  return acc;
}

// S_F,K (uF = u.F; uf = 2 u_x F_x, 2 u_y F_y, 2 u_z F_z, u_x F_y + u_y F_x,
// u_y F_z + u_z F_y, u_x F_z + u_z F_x)
template <int Q, int K, typename V, typename R>
__host__ __device__ __forceinline__ V moment_source(V uF, R Fx, R Fy, R Fz, const V* uf) {
  constexpr double A = -3.0 * eq_a<Q>(K);
  constexpr double Bx = 3.0 * eq_b<Q>(K, 0), By = 3.0 * eq_b<Q>(K, 1), Bz = 3.0 * eq_b<Q>(K, 2);
  constexpr double Cxx = 4.5 * eq_c<Q>(K, 0, 0), Cyy = 4.5 * eq_c<Q>(K, 1, 1),
                   Czz = 4.5 * eq_c<Q>(K, 2, 2), Cxy = 9.0 * eq_c<Q>(K, 0, 1),
                   Cyz = 9.0 * eq_c<Q>(K, 1, 2), Cxz = 9.0 * eq_c<Q>(K, 0, 2);
  R b = R(0);  // the constant part, in the arithmetic type
  if constexpr (Bx != 0.0) b += R(Bx) * Fx;
  if constexpr (By != 0.0) b += R(By) * Fy;
  if constexpr (Bz != 0.0) b += R(Bz) * Fz;
  V acc = V(b);
  acc = add_scaled<V, R>(acc, A, uF);
  acc = add_scaled<V, R>(acc, Cxx, uf[0]);
  acc = add_scaled<V, R>(acc, Cyy, uf[1]);
  acc = add_scaled<V, R>(acc, Czz, uf[2]);
  acc = add_scaled<V, R>(acc, Cxy, uf[3]);
  acc = add_scaled<V, R>(acc, Cyz, uf[4]);
  acc = add_scaled<V, R>(acc, Cxz, uf[5]);
  return acc;
}

}  // namespace lbm
