// Non-equilibrium extrapolation of one boundary node (see lbm_neq.cu), a
// host/device function so that host builds of the kernel code can run it.
#pragma once

#include "lbm_kernels.cuh"

namespace lbm {

struct NeqArgs {
  int vel, pre;         // face bits of the velocity / pressure faces
  int off[7];           // prefix of the boundary-plane sizes, face by face
  double pb[6];         // pressure of each pressure face at this time level
};

__host__ __device__ inline int face_axis(int f) { return f >> 1; }

// Extrapolation of boundary index t (0 <= t < a.off[6]); indices of the
// face planes in order, x fastest within a plane; a node on several
// extrapolation planes is handled by the index of its first plane only.
template <int Q, typename S, typename R, bool ODD>
__host__ __device__ inline void neq_node(const Domain<R>& d, const NeqArgs& a, int t) {
  int face = 0;
  while (face < 5 && t >= a.off[face + 1]) ++face;
  const int local = t - a.off[face];
  // node of plane `face`: the two in-plane axes in order, x fastest
  const int k = face_axis(face);
  const int n[3] = {d.nx, d.ny, d.nz};
  const int u_ax = k == 0 ? 1 : 0, v_ax = k == 2 ? 1 : 2;
  int xyz[3];
  xyz[k] = (face & 1) ? n[k] - 1 : 0;
  xyz[u_ax] = local % n[u_ax];
  xyz[v_ax] = local / n[u_ax];
  const int neq = a.vel | a.pre;
  // the faces of the node; a node on several planes belongs to the first
  int xf[3] = {xyz[0], xyz[1], xyz[2]};
  int vel_face = -1, pre_face = -1;
#pragma unroll
  for (int g = 0; g < 6; ++g) {
    const int ax = face_axis(g);
    const bool on = (g & 1) ? xyz[ax] == n[ax] - 1 : xyz[ax] == 0;
    if (!on || !((neq >> g) & 1)) continue;
    if (g < face) return;  // handled by the thread of plane g
    xf[ax] = (g & 1) ? n[ax] - 2 : 1;
    if (((a.vel >> g) & 1) && vel_face < 0) vel_face = g;
    if (((a.pre >> g) & 1) && pre_face < 0) pre_face = g;
  }
  R fv[Q];
  get_canonical<Q, S, R, ODD>(d, static_cast<const S*>(d.f), xf[0], xf[1], xf[2], fv);
  R P = R(0), uf[3] = {R(0), R(0), R(0)};
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    P += fv[q];
    uf[0] += R(Lattice<Q>::c(q, 0)) * fv[q];
    uf[1] += R(Lattice<Q>::c(q, 1)) * fv[q];
    uf[2] += R(Lattice<Q>::c(q, 2)) * fv[q];
  }
  for (int c = 0; c < 3; ++c) uf[c] += R(0.5) * d.F[c];
  // Eq. hgl: p = c_s^2 / (1 - w0) (P - w0 |u|^2 / (2 c_s^2)), c_s^2 = 1/3
  constexpr double w0 = Lattice<Q>::w0;
  const R uf2 = uf[0] * uf[0] + uf[1] * uf[1] + uf[2] * uf[2];
  const R pf = R(1.0 / (3.0 * (1.0 - w0))) * (P - R(1.5 * w0) * uf2);
  R ub[3], pb;
  for (int c = 0; c < 3; ++c) ub[c] = vel_face >= 0 ? d.uw[vel_face][c] : uf[c];
  pb = pre_face >= 0 ? R(a.pb[pre_face]) : pf;
  const R ub2 = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const R cx = R(Lattice<Q>::c(q, 0)), cy = R(Lattice<Q>::c(q, 1)), cz = R(Lattice<Q>::c(q, 2));
    const R w = R(Lattice<Q>::w(q));
    const R cub = cx * ub[0] + cy * ub[1] + cz * ub[2];
    const R cuf = cx * uf[0] + cy * uf[1] + cz * uf[2];
    // Eq. edf: f_eq = w (3 p + 3 c.u + 9/2 (c.u)^2 - 3/2 |u|^2)
    const R eb = w * (R(3) * pb + R(3) * cub + R(4.5) * cub * cub - R(1.5) * ub2);
    const R ef = w * (R(3) * pf + R(3) * cuf + R(4.5) * cuf * cuf - R(1.5) * uf2);
    fv[q] = eb + (fv[q] - ef);
  }
  put_canonical<Q, S, R, ODD>(d, static_cast<S*>(d.f), xyz[0], xyz[1], xyz[2], fv);
}

}  // namespace lbm
