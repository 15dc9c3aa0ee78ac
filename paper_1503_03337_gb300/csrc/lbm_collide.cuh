// One-cell MRT collision, Eq. mrteqvT:
//   f* = f - T^-1 [ S (m - m_eq) - (I - S/2) S_F ]
//
// u = j + F/2 and p from Eq. hgl.  The Guo source S_F is the derivative of
// the equilibrium moments along F at fixed p (the first-order rows give F,
// the quadratic ones 2 B(u, F) for m_eq = B(u, u)); its P row is zero, so P
// stays a collision invariant.  Because p is computed from P, P - P_eq = 0
// exactly and j - u = -F/2, so the conserved rows contribute only -F to the
// momentum rows whatever s_c is.
//
// Every model uses the factored transforms of lbm_factored.cuh; iD3Q14 and
// iD3Q18 the printed closed-form equilibria, iD3Q26 m_eq = T f_eq
// (moment_eq).
// On return f holds f*, and (ux,uy,uz) the velocity of the pre-collision
// state.  V is the value type (float, double, or pf2 for two cells at once)
// and R the scalar type of rates, force and constants.
#pragma once

#include "lbm_factored.cuh"
#include "lbm_model.cuh"

namespace lbm {

// Velocity, pressure and the products the equilibria and sources need.
template <int Q, bool FORCE, typename V, typename R>
struct CellState {
  V ux, uy, uz, u2, p;
  V uxx, uyy, uzz, uxy, uyz, uxz;
  // force terms (zero without FORCE): u.F, 6 u_x F_x - 2 u.F,
  // 2 (u_y F_y - u_z F_z), u_x F_y + u_y F_x, u_y F_z + u_z F_y, u_x F_z + u_z F_x
  V uF, sxx, sww, sxy, syz, sxz;

  __host__ __device__ __forceinline__ CellState(V P, V jx, V jy, V jz, R Fx, R Fy, R Fz) {
    if constexpr (FORCE) {
      ux = jx + R(0.5) * Fx;
      uy = jy + R(0.5) * Fy;
      uz = jz + R(0.5) * Fz;
    } else {
      ux = jx;
      uy = jy;
      uz = jz;
    }
    uxx = ux * ux;
    uyy = uy * uy;
    uzz = uz * uz;
    u2 = uxx + uyy + uzz;
    constexpr double cs2 = 1.0 / 3.0;
    constexpr double w0 = Lattice<Q>::w0;
    p = R(cs2 / (1.0 - w0)) * (P - R(w0 / (2.0 * cs2)) * u2);
    uxy = ux * uy;
    uyz = uy * uz;
    uxz = ux * uz;
    uF = sxx = sww = sxy = syz = sxz = V(R(0));
    if constexpr (FORCE) {
      uF = ux * Fx + uy * Fy + uz * Fz;
      sxx = R(6) * ux * Fx - R(2) * uF;
      sww = R(2) * (uy * Fy - uz * Fz);
      sxy = ux * Fy + uy * Fx;
      syz = uy * Fz + uz * Fy;
      sxz = ux * Fz + uz * Fx;
    }
  }
};

// Pair sums and differences s_I = f_rep + f_opp, d_I = f_rep - f_opp.
template <int Q, typename V>
__host__ __device__ __forceinline__ void pair_split(const V* f, V* ps, V* pd) {
  [&]<int... I>(std::integer_sequence<int, I...>) {
    ((ps[I] = f[pair_rep<Q>(I)] + f[opposite<Q>(pair_rep<Q>(I))],
      pd[I] = f[pair_rep<Q>(I)] - f[opposite<Q>(pair_rep<Q>(I))]),
     ...);
  }(std::make_integer_sequence<int, Q / 2>{});
}

// iD3Q14 / iD3Q18 with the factored transforms.  f* = T' D^-1 m* is formed
// from every post-collision row y_K = m*_K / D_K = g_K m_K + k_K m_eq,K +
// h_K S_F,K, so the populations and pair sums are dead once the moments are
// known.  The conserved rows give y_0 = P / D_0 and y_j = (j + F) / D_j
// (m*_j = j + F whatever s_c is, because m_eq,j = u = j + F/2 and S_F,j = F).
template <int Q, bool FORCE, typename V, typename R>
__host__ __device__ __forceinline__ void collide_factored(V* f, const Rates<R>& s, R Fx, R Fy,
                                                          R Fz, V& ux, V& uy, V& uz) {
  static_assert(Q == 14 || Q == 18, "factored transforms exist for iD3Q14 and iD3Q18");
  constexpr int NP = Q / 2;
  V m[Q];
  {
    V ps[NP], pd[NP];
    pair_split<Q>(f, ps, pd);
    Factored<Q>::moments(ps, pd, m);
  }
  const CellState<Q, FORCE, V, R> c(m[0], m[2], m[4], m[6], Fx, Fy, Fz);
  ux = c.ux;
  uy = c.uy;
  uz = c.uz;

  V* y = m;  // y_K replaces m_K
  y[0] = R(1.0 / row_norm<Q>(0)) * m[0];
  if constexpr (FORCE) {
    y[2] = R(1.0 / row_norm<Q>(2)) * (m[2] + Fx);
    y[4] = R(1.0 / row_norm<Q>(4)) * (m[4] + Fy);
    y[6] = R(1.0 / row_norm<Q>(6)) * (m[6] + Fz);
  } else {
    y[2] = R(1.0 / row_norm<Q>(2)) * m[2];
    y[4] = R(1.0 / row_norm<Q>(4)) * m[4];
    y[6] = R(1.0 / row_norm<Q>(6)) * m[6];
  }
  // a relaxed row: g m + k m_eq (+ h S_F)
  auto relax = [&](int K, V meq) { return fmadd(V(s.k[K]), meq, s.g[K] * m[K]); };
  auto source = [&](int K, V v, V src) { return fmadd(V(s.h[K]), src, v); };
  const V pxx_eq = R(3) * c.uxx - c.u2;  // 3 p_xx
  const V pww_eq = c.uyy - c.uzz;
  if constexpr (Q == 14) {
    y[1] = relax(1, R(-7) * c.p + c.u2);  // e_eq = -7p + u^2, source 2 u.F
    if constexpr (FORCE) y[1] = source(1, y[1], R(2) * c.uF);
  } else {
    y[1] = relax(1, R(0.5) * c.u2 - c.p);  // e_eq = -p + u^2/2, source u.F
    if constexpr (FORCE) y[1] = source(1, y[1], c.uF);
  }
  // q_eq = -cq u with cq = 7/3 (Q14) or 2/3 (Q18); source -cq F
  constexpr double cq = Q == 14 ? 7.0 / 3.0 : 2.0 / 3.0;
  y[3] = relax(3, R(-cq) * c.ux);
  y[5] = relax(5, R(-cq) * c.uy);
  y[7] = relax(7, R(-cq) * c.uz);
  if constexpr (FORCE) {
    y[3] = source(3, y[3], V(R(-cq) * Fx));
    y[5] = source(5, y[5], V(R(-cq) * Fy));
    y[7] = source(7, y[7], V(R(-cq) * Fz));
  }
  y[8] = relax(8, pxx_eq);
  if constexpr (FORCE) y[8] = source(8, y[8], c.sxx);
  if constexpr (Q == 14) {
    y[9] = relax(9, pww_eq);
    y[10] = relax(10, c.uxy);
    y[11] = relax(11, c.uyz);
    y[12] = relax(12, c.uxz);
    if constexpr (FORCE) {
      y[9] = source(9, y[9], c.sww);
      y[10] = source(10, y[10], c.sxy);
      y[11] = source(11, y[11], c.syz);
      y[12] = source(12, y[12], c.sxz);
    }
    y[13] = s.g[13] * m[13];
  } else {
    // 3pi_xx and pi_ww equilibria (and sources) are -1/2 of 3p_xx and p_ww
    y[9] = relax(9, R(-0.5) * pxx_eq);
    y[10] = relax(10, pww_eq);
    y[11] = relax(11, R(-0.5) * pww_eq);
    y[12] = relax(12, c.uxy);
    y[13] = relax(13, c.uyz);
    y[14] = relax(14, c.uxz);
    if constexpr (FORCE) {
      y[9] = source(9, y[9], R(-0.5) * c.sxx);
      y[10] = source(10, y[10], c.sww);
      y[11] = source(11, y[11], R(-0.5) * c.sww);
      y[12] = source(12, y[12], c.sxy);
      y[13] = source(13, y[13], c.syz);
      y[14] = source(14, y[14], c.sxz);
    }
    y[15] = s.g[15] * m[15];
    y[16] = s.g[16] * m[16];
    y[17] = s.g[17] * m[17];
  }

  V C[NP], D[NP];
  Factored<Q>::cols_even(y, C);
  Factored<Q>::cols_odd(y, D);
  [&]<int... I>(std::integer_sequence<int, I...>) {
    ((f[pair_rep<Q>(I)] = C[I] + D[I], f[opposite<Q>(pair_rep<Q>(I))] = C[I] - D[I]), ...);
  }(std::make_integer_sequence<int, NP>{});
}

// A model without printed equilibria (iD3Q26): the factored transforms, and
// every post-collision row y_K = m*_K / D_K with the equilibrium moments and
// sources from their definition m_eq = T f_eq (moment_eq, moment_source).
// As in collide_factored, the pair sums are dead once the moments are known.
template <int Q, bool FORCE, typename V, typename R>
__host__ __device__ __forceinline__ void collide_teq(V* f, const Rates<R>& s, R Fx, R Fy, R Fz,
                                                     V& ux, V& uy, V& uz) {
  constexpr int NP = Q / 2;
  V m[Q];
  {
    V ps[NP], pd[NP];
    pair_split<Q>(f, ps, pd);
    Factored<Q>::moments(ps, pd, m);
  }
  const CellState<Q, FORCE, V, R> c(m[0], m[2], m[4], m[6], Fx, Fy, Fz);
  ux = c.ux;
  uy = c.uy;
  uz = c.uz;
  const V q3 = R(3) * c.p - R(1.5) * c.u2;
  const V uu[6] = {c.uxx, c.uyy, c.uzz, c.uxy, c.uyz, c.uxz};
  V uf[6] = {V(R(0)), V(R(0)), V(R(0)), V(R(0)), V(R(0)), V(R(0))};
  if constexpr (FORCE) {
    uf[0] = R(2) * (c.ux * Fx);
    uf[1] = R(2) * (c.uy * Fy);
    uf[2] = R(2) * (c.uz * Fz);
    uf[3] = c.sxy;
    uf[4] = c.syz;
    uf[5] = c.sxz;
  }
  V* y = m;  // y_K replaces m_K
  y[0] = R(1.0 / row_norm<Q>(0)) * m[0];
  if constexpr (FORCE) {  // m*_j = j + F (see collide_factored)
    y[2] = R(1.0 / row_norm<Q>(2)) * (m[2] + Fx);
    y[4] = R(1.0 / row_norm<Q>(4)) * (m[4] + Fy);
    y[6] = R(1.0 / row_norm<Q>(6)) * (m[6] + Fz);
  } else {
    y[2] = R(1.0 / row_norm<Q>(2)) * m[2];
    y[4] = R(1.0 / row_norm<Q>(4)) * m[4];
    y[6] = R(1.0 / row_norm<Q>(6)) * m[6];
  }
  auto relax = [&]<int K>() {
    V v = fmadd(V(s.k[K]), moment_eq<Q, K, V, R>(q3, c.ux, c.uy, c.uz, uu), s.g[K] * m[K]);
    if constexpr (FORCE) v = fmadd(V(s.h[K]), moment_source<Q, K, V, R>(c.uF, Fx, Fy, Fz, uf), v);
    y[K] = v;
  };
  relax.template operator()<1>();
  relax.template operator()<3>();
  relax.template operator()<5>();
  [&]<int... K>(std::integer_sequence<int, K...>) {
    (relax.template operator()<K + 7>(), ...);
  }(std::make_integer_sequence<int, Q - 7>{});
  V C[NP], D[NP];
  Factored<Q>::cols_even(y, C);
  Factored<Q>::cols_odd(y, D);
  [&]<int... I>(std::integer_sequence<int, I...>) {
    ((f[pair_rep<Q>(I)] = C[I] + D[I], f[opposite<Q>(pair_rep<Q>(I))] = C[I] - D[I]), ...);
  }(std::make_integer_sequence<int, NP>{});
}

template <int Q, bool FORCE, typename V, typename R>
__host__ __device__ __forceinline__ void collide(V* f, const Rates<R>& s, R Fx, R Fy, R Fz,
                                                 V& ux, V& uy, V& uz) {
  if constexpr (Q == 14 || Q == 18) collide_factored<Q, FORCE>(f, s, Fx, Fy, Fz, ux, uy, uz);
  else collide_teq<Q, FORCE>(f, s, Fx, Fy, Fz, ux, uy, uz);
}

}  // namespace lbm
