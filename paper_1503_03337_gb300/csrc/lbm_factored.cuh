// Factored moment transforms of iD3Q14 (Sec. 3), iD3Q18 (App. B) and iD3Q26.
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

template <>
struct Factored<26> {
  // rows: the 18 of iD3Q18, then |c|^4, |c|^4 c_x, |c|^4 c_y, |c|^4 c_z,
  // |c|^2 c_x c_y, |c|^2 c_y c_z, |c|^2 c_x c_z, c_x c_y c_z (phi<26>).
  // Pairs 0-8 are those of iD3Q18 (axes, face diagonals), pairs 9-12 the
  // cube diagonals (1,1,1) (-1,1,1) (1,-1,1) (-1,-1,1).  Each row is a shell
  // polynomial times a monomial, so it is a combination of the axis, face
  // and cube partial sums of that monomial.
  template <typename V>
  __host__ __device__ __forceinline__ static constexpr void moments(const V* s, const V* d,
                                                                    V* m) {
    // even rows
    const V Y = s[1] + s[2];
    const V A = s[0] + Y;                     // axes
    const V a = s[3] + s[4], b = s[5] + s[6], c = s[7] + s[8];
    const V ab = a + b;
    const V B = ab + c;                       // face diagonals
    const V u1 = s[9] + s[10], u2 = s[11] + s[12], v1 = s[9] - s[10], v2 = s[11] - s[12];
    const V K = u1 + u2;                      // cube diagonals
    m[0] = A + B + K;
    m[1] = term_add<12>(term_add<-14>(-B, A), K);   // -14, -1, 12 on the shells
    m[18] = term_add<3>(V(4) * (A - B), K);                // 4, -4, 3
    const V X = term_add<-2>(ab, c);
    m[8] = term_add<2>(X - Y, s[0]);
    m[9] = term_add<-4>(term_add<2>(X, Y), s[0]);
    const V W1 = s[1] - s[2], W2 = a - b;
    m[10] = W1 + W2;
    m[11] = term_add<-2>(W2, W1);
    // c_x c_y, c_y c_z, c_x c_z on faces (F) and cube (Kc); the |c|^2
    // weighted rows take -2 on the faces and 1 on the cube
    const V Fxy = s[3] - s[4], Fyz = s[7] - s[8], Fxz = s[5] - s[6];
    const V Kxy = v1 - v2, Kyz = u1 - u2, Kxz = v1 + v2;
    m[12] = Fxy + Kxy;
    m[13] = Fyz + Kyz;
    m[14] = Fxz + Kxz;
    m[22] = term_add<-2>(Kxy, Fxy);
    m[23] = term_add<-2>(Kyz, Fyz);
    m[24] = term_add<-2>(Kxz, Fxz);
    // odd rows: face and cube partial sums of c_x, c_y, c_z
    const V x1 = d[3] - d[4], x2 = d[5] - d[6];
    const V y1 = d[3] + d[4], y2 = d[7] - d[8];
    const V z1 = d[5] + d[6], z2 = d[7] + d[8];
    const V Fx = x1 + x2, Fy = y1 + y2, Fz = z1 + z2;
    m[15] = x1 - x2;
    m[16] = y2 - y1;
    m[17] = z1 - z2;
    const V p1 = d[9] + d[10], p2 = d[11] + d[12], q1 = d[9] - d[10], q2 = d[11] - d[12];
    const V Kx = q1 + q2, Ky = p1 - p2, Kz = p1 + p2;
    m[25] = q1 - q2;
    // j: 1, 1, 1; q = (3|c|^2 - 7) c: -4, -1, 2; |c|^4 c row: 4, -2, 1
    m[2] = d[0] + Fx + Kx;
    m[3] = term_add<2>(term_add<-4>(-Fx, d[0]), Kx);
    m[19] = term_add<-2>(term_add<4>(Kx, d[0]), Fx);
    m[4] = d[1] + Fy + Ky;
    m[5] = term_add<2>(term_add<-4>(-Fy, d[1]), Ky);
    m[20] = term_add<-2>(term_add<4>(Ky, d[1]), Fy);
    m[6] = d[2] + Fz + Kz;
    m[7] = term_add<2>(term_add<-4>(-Fz, d[2]), Kz);
    m[21] = term_add<-2>(term_add<4>(Kz, d[2]), Fz);
  }

  template <typename V>
  __host__ __device__ __forceinline__ static constexpr void cols_even(const V* x, V* C) {
    // axes: P - 14 e + 4 |c|^4, then as iD3Q18
    const V Ax = term_add<4>(term_add<-14>(x[0], x[1]), x[18]);
    C[0] = term_add<-4>(term_add<2>(Ax, x[8]), x[9]);
    const V G = term_add<2>(Ax - x[8], x[9]);
    const V Wv = term_add<-2>(x[10], x[11]);
    C[1] = G + Wv;
    C[2] = G - Wv;
    // face diagonals: P - e - 4 |c|^4, then as iD3Q18, and the c_x c_y
    // rows with 1 (plain) and -2 (|c|^2 weighted)
    const V Fc = term_add<-4>(x[0] - x[1], x[18]);
    const V T = x[8] + x[9];
    const V U = Fc + T;
    const V W = x[10] + x[11];
    const V Cxy = U + W, Cxz = U - W;
    const V Cyz = term_add<-2>(Fc, T);
    const V Pxy = term_add<-2>(x[12], x[22]), Pyz = term_add<-2>(x[13], x[23]),
            Pxz = term_add<-2>(x[14], x[24]);
    C[3] = Cxy + Pxy;
    C[4] = Cxy - Pxy;
    C[5] = Cxz + Pxz;
    C[6] = Cxz - Pxz;
    C[7] = Cyz + Pyz;
    C[8] = Cyz - Pyz;
    // cube diagonals: P + 12 e + 3 |c|^4 and the c_x c_y rows with 1 and 1
    const V Kc = term_add<3>(term_add<12>(x[0], x[1]), x[18]);
    const V Qxy = x[12] + x[22], Qyz = x[13] + x[23], Qxz = x[14] + x[24];
    const V gp = Qxy + Qxz, gm = Qxy - Qxz, hp = Kc + Qyz, hm = Kc - Qyz;
    C[9] = hp + gp;
    C[10] = hp - gp;
    C[11] = hm - gm;
    C[12] = hm + gm;
  }

  template <typename V>
  __host__ __device__ __forceinline__ static constexpr void cols_odd(const V* x, V* D) {
    // per axis, j + q + |c|^4 c on the three shells: 1 - 4 + 4 on the
    // axis, 1 - 1 - 2 on the faces, 1 + 2 + 1 on the cube
    D[0] = term_add<4>(term_add<-4>(x[2], x[3]), x[19]);
    D[1] = term_add<4>(term_add<-4>(x[4], x[5]), x[20]);
    D[2] = term_add<4>(term_add<-4>(x[6], x[7]), x[21]);
    const V Gx = term_add<-2>(x[2] - x[3], x[19]), Gy = term_add<-2>(x[4] - x[5], x[20]),
            Gz = term_add<-2>(x[6] - x[7], x[21]);
    const V a1 = Gx + x[15], b1 = Gy - x[16];
    D[3] = a1 + b1;
    D[4] = b1 - a1;
    const V a2 = Gx - x[15], b2 = Gz + x[17];
    D[5] = a2 + b2;
    D[6] = b2 - a2;
    const V a3 = Gy + x[16], b3 = Gz - x[17];
    D[7] = a3 + b3;
    D[8] = b3 - a3;
    const V Hx = term_add<2>(x[2] + x[19], x[3]), Hy = term_add<2>(x[4] + x[20], x[5]),
            Hz = term_add<2>(x[6] + x[21], x[7]);
    const V zp = Hz + x[25], zm = Hz - x[25];
    const V sxy = Hx + Hy, dxy = Hy - Hx;
    D[9] = zp + sxy;
    D[10] = zm + dxy;
    D[11] = zm - dxy;
    D[12] = zp - sxy;
  }
};
// The factored functions against T, on integer unit vectors (phi and the
// pair representatives tabulated once, to stay within the compiler's
// constant-evaluation budget).
template <int Q>
constexpr bool factored_ok() {
  constexpr int NP = Q / 2;
  int t[Q][NP] = {};
  bool even[Q] = {};
  for (int I = 0; I < NP; ++I) {
    const int rep = pair_rep<Q>(I);
    for (int K = 0; K < Q; ++K) t[K][I] = phi<Q>(K, rep);
  }
  for (int K = 0; K < Q; ++K) even[K] = row_even<Q>(K);
  for (int I = 0; I < NP; ++I) {
    for (int odd = 0; odd < 2; ++odd) {
      int s[NP] = {}, d[NP] = {}, m[Q] = {};
      (odd ? d : s)[I] = 1;
      Factored<Q>::moments(s, d, m);
      for (int K = 0; K < Q; ++K)
        if (m[K] != (even[K] != (odd != 0) ? t[K][I] : 0)) return false;
    }
  }
  for (int K = 0; K < Q; ++K) {
    int x[Q] = {}, C[NP] = {}, D[NP] = {};
    x[K] = 1;
    Factored<Q>::cols_even(x, C);
    Factored<Q>::cols_odd(x, D);
    for (int I = 0; I < NP; ++I) {
      if (C[I] != (even[K] ? t[K][I] : 0)) return false;
      if (D[I] != (even[K] ? 0 : t[K][I])) return false;
    }
  }
  return true;
}
static_assert(factored_ok<14>(), "iD3Q14 factored transform differs from T");
static_assert(factored_ok<18>(), "iD3Q18 factored transform differs from T");
static_assert(factored_ok<26>(), "iD3Q26 factored transform differs from T");

}  // namespace lbm
