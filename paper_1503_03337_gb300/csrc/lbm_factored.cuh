// Factored moment transforms of iD3Q14 (Sec. 3) and iD3Q18 (App. B).
//
// m = T f runs on the opposite-pair sums s_I (even rows) and differences d_I
// (odd rows).  Evaluated row by row, each row is its own chain of adds: the
// compiler may not reassociate floating-point sums, so rows that share
// partial sums (the face diagonals of one plane, the cube diagonals, the
// axes) recompute them.  Here the shared sums are written out once:
//   iD3Q18: moments 78 -> 40 operations, back-transform columns 81 -> 42;
//   iD3Q14: moments 51 -> 29, columns 49 -> 31.
// The back-transform f* = T' D^-1 m* needs, per pair I, the even and odd
// column sums
//   C_I = sum over even rows K of phi_K(rep_I) y_K,
//   D_I = sum over odd rows K of phi_K(rep_I) y_K,
// with y_K = m*_K / D_K the post-collision row divided by its norm; then
//   f*_rep = C_I + D_I,  f*_opp = C_I - D_I.
// Every function is a template on the value type so that factored_ok<Q>()
// can evaluate it on integer unit vectors at compile time: it proves that
// the moments equal T (on s and d) and the columns equal T' exactly.
//
// Pair index I (pair_rep order, checked by factored_ok):
//   iD3Q18: (1,0,0) (0,1,0) (0,0,1) (1,1,0) (-1,1,0) (1,0,1) (-1,0,1) (0,1,1) (0,-1,1)
//   iD3Q14: (1,0,0) (0,1,0) (0,0,1) (1,1,1) (-1,1,1) (1,-1,1) (-1,-1,1)
#pragma once

#include "lbm_model.cuh"  // basis, rows, term helpers

namespace lbm {

template <int Q>
struct Factored;

template <>
struct Factored<18> {
  // rows: P, e, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz,
  // pxz, tx, ty, tz
  template <typename V>
  __host__ __device__ __forceinline__ static constexpr void moments(const V* s, const V* d,
                                                                    V* m) {
    // even rows: sums of the xy, xz and yz face-diagonal pairs and of the
    // y and z axes
    const V a = s[3] + s[4], b = s[5] + s[6], c = s[7] + s[8];
    const V Y = s[1] + s[2];
    const V A = s[0] + Y;           // axes
    const V ab = a + b;
    const V B = ab + c;             // face diagonals
    m[0] = A + B;                   // P
    m[1] = term_add<-2>(B, A);      // e: -2 on the axes, 1 on the diagonals
    const V X = term_add<-2>(ab, c);
    m[8] = term_add<2>(X - Y, s[0]);                // 2 s0 - s1 - s2 + a + b - 2c
    m[9] = term_add<-4>(term_add<2>(X, Y), s[0]);   // -4 s0 + 2 s1 + 2 s2 + a + b - 2c
    const V W1 = s[1] - s[2], W2 = a - b;
    m[10] = W1 + W2;                // s1 - s2 + a - b
    m[11] = term_add<-2>(W2, W1);   // -2 s1 + 2 s2 + a - b
    m[12] = s[3] - s[4];
    m[13] = s[7] - s[8];
    m[14] = s[5] - s[6];
    // odd rows: along each axis, the two face-diagonal planes through it
    const V x1 = d[3] - d[4], x2 = d[5] - d[6];
    const V Dx = x1 + x2;
    m[2] = d[0] + Dx;
    m[3] = term_add<-4>(Dx, d[0]);
    m[15] = x1 - x2;
    const V y1 = d[3] + d[4], y2 = d[7] - d[8];
    const V Dy = y1 + y2;
    m[4] = d[1] + Dy;
    m[5] = term_add<-4>(Dy, d[1]);
    m[16] = y2 - y1;
    const V z1 = d[5] + d[6], z2 = d[7] + d[8];
    const V Dz = z1 + z2;
    m[6] = d[2] + Dz;
    m[7] = term_add<-4>(Dz, d[2]);
    m[17] = z1 - z2;
  }

  template <typename V>
  __host__ __device__ __forceinline__ static constexpr void cols_even(const V* x, V* C) {
    const V T = x[8] + x[9];
    const V P1 = x[0] + x[1];
    const V U = P1 + T;  // P + e + 3pxx + 3pixx on the xy and xz diagonals
    const V W = x[10] + x[11];
    const V Cxy = U + W, Cxz = U - W;
    C[3] = Cxy + x[12];
    C[4] = Cxy - x[12];
    C[5] = Cxz + x[14];
    C[6] = Cxz - x[14];
    const V Cyz = term_add<-2>(P1, T);
    C[7] = Cyz + x[13];
    C[8] = Cyz - x[13];
    // axes: P - 2 e, then -3pxx + 2 3pixx (+-) (pww - 2 piww) on y and z,
    // 2 3pxx - 4 3pixx on x
    const V A = term_add<-2>(x[0], x[1]);
    const V G = term_add<2>(A - x[8], x[9]);
    const V Wv = term_add<-2>(x[10], x[11]);
    C[1] = G + Wv;
    C[2] = G - Wv;
    C[0] = term_add<-4>(term_add<2>(A, x[8]), x[9]);
  }

  template <typename V>
  __host__ __device__ __forceinline__ static constexpr void cols_odd(const V* x, V* D) {
    // on a diagonal, j and q of an axis both enter as c_axis
    const V Gx = x[2] + x[3], Gy = x[4] + x[5], Gz = x[6] + x[7];
    D[0] = term_add<-4>(x[2], x[3]);
    D[1] = term_add<-4>(x[4], x[5]);
    D[2] = term_add<-4>(x[6], x[7]);
    const V a1 = Gx + x[15], b1 = Gy - x[16];
    D[3] = a1 + b1;
    D[4] = b1 - a1;
    const V a2 = Gx - x[15], b2 = Gz + x[17];
    D[5] = a2 + b2;
    D[6] = b2 - a2;
    const V a3 = Gy + x[16], b3 = Gz - x[17];
    D[7] = a3 + b3;
    D[8] = b3 - a3;
  }
};

template <>
struct Factored<14> {
  // rows: P, e, jx, qx, jy, qy, jz, qz, 3pxx, pww, pxy, pyz, pxz, txyz
  template <typename V>
  __host__ __device__ __forceinline__ static constexpr void moments(const V* s, const V* d,
                                                                    V* m) {
    const V Y = s[1] + s[2];
    const V A = s[0] + Y;  // axes
    // the four cube-diagonal pairs, combined two by two
    const V u1 = s[3] + s[4], u2 = s[5] + s[6], v1 = s[3] - s[4], v2 = s[5] - s[6];
    const V B = u1 + u2;
    m[0] = A + B;
    m[1] = term_add<3>(V(-4) * A, B);  // e: -4 on the axes, 3 on the diagonals
    m[8] = V(2) * s[0] - Y;
    m[9] = s[1] - s[2];
    m[10] = v1 - v2;
    m[11] = u1 - u2;
    m[12] = v1 + v2;
    const V p1 = d[3] + d[4], p2 = d[5] + d[6], q1 = d[3] - d[4], q2 = d[5] - d[6];
    const V Dx = q1 + q2, Dy = p1 - p2, Dz = p1 + p2;
    m[2] = d[0] + Dx;
    m[3] = term_add<-4>(Dx, d[0]);
    m[4] = d[1] + Dy;
    m[5] = term_add<-4>(Dy, d[1]);
    m[6] = d[2] + Dz;
    m[7] = term_add<-4>(Dz, d[2]);
    m[13] = q1 - q2;
  }

  template <typename V>
  __host__ __device__ __forceinline__ static constexpr void cols_even(const V* x, V* C) {
    const V n4 = term_add<-4>(x[0], x[1]);  // P - 4 e on the axes
    C[0] = term_add<2>(n4, x[8]);
    C[1] = n4 + (x[9] - x[8]);
    C[2] = n4 - (x[8] + x[9]);
    const V e3 = term_add<3>(x[0], x[1]);   // P + 3 e on the diagonals
    const V gp = x[10] + x[12], gm = x[10] - x[12];
    const V hp = e3 + x[11], hm = e3 - x[11];
    C[3] = hp + gp;
    C[4] = hp - gp;
    C[5] = hm - gm;
    C[6] = hm + gm;
  }

  template <typename V>
  __host__ __device__ __forceinline__ static constexpr void cols_odd(const V* x, V* D) {
    const V Gx = x[2] + x[3], Gy = x[4] + x[5], Gz = x[6] + x[7];
    D[0] = term_add<-4>(x[2], x[3]);
    D[1] = term_add<-4>(x[4], x[5]);
    D[2] = term_add<-4>(x[6], x[7]);
    const V zp = Gz + x[13], zm = Gz - x[13];
    const V sxy = Gx + Gy, dxy = Gy - Gx;
    D[3] = zp + sxy;
    D[4] = zm + dxy;
    D[5] = zm - dxy;
    D[6] = zp - sxy;
  }
};

// The factored functions against T, on integer unit vectors.
template <int Q>
constexpr bool factored_ok() {
  constexpr int NP = Q / 2;
  for (int I = 0; I < NP; ++I) {
    for (int odd = 0; odd < 2; ++odd) {
      int s[NP] = {}, d[NP] = {}, m[Q] = {};
      (odd ? d : s)[I] = 1;
      Factored<Q>::moments(s, d, m);
      for (int K = 0; K < Q; ++K) {
        const bool use = row_even<Q>(K) != (odd != 0);
        if (m[K] != (use ? phi<Q>(K, pair_rep<Q>(I)) : 0)) return false;
      }
    }
  }
  for (int K = 0; K < Q; ++K) {
    int x[Q] = {}, C[NP] = {}, D[NP] = {};
    x[K] = 1;
    Factored<Q>::cols_even(x, C);
    Factored<Q>::cols_odd(x, D);
    const bool even = row_even<Q>(K);
    for (int I = 0; I < NP; ++I) {
      const int t = phi<Q>(K, pair_rep<Q>(I));
      if (C[I] != (even ? t : 0)) return false;
      if (D[I] != (even ? 0 : t)) return false;
    }
  }
  return true;
}
static_assert(factored_ok<14>(), "iD3Q14 factored transform differs from T");
static_assert(factored_ok<18>(), "iD3Q18 factored transform differs from T");

}  // namespace lbm
