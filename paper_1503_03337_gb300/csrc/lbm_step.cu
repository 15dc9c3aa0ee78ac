// Single-domain step: descriptor conversion, force time level, default launch
// shape, and dispatch to the per-Q kernel files (lbm_step_q14.cu, _q18.cu,
// _q26.cu).
#include <cmath>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

template <typename R>
Domain<R> to_domain(const DomainDesc& d, const double F[3]) {
  Domain<R> o{};
  o.f = d.f;
  o.nx = d.nx;
  o.ny = d.ny;
  o.nz = d.nz;
  o.N = d.N;
  for (int k = 0; k < 3; ++k) o.per[k] = d.per[k];
  o.moving = d.moving;
  o.sym = d.sym;
  o.solid = d.solid;
  for (int face = 0; face < 6; ++face) {
    for (int k = 0; k < 3; ++k) o.uw[face][k] = R(d.uw[face][k]);
    o.edge_axis[face] = d.edge_axis[face];
    for (int k = 0; k < 2; ++k) o.edge_scale[face][k] = R(d.edge_scale[face][k]);
  }
  o.s.sc = R(d.s[0]);
  o.s.se = R(d.s[1]);
  o.s.sq = R(d.s[2]);
  o.s.snu = R(d.s[3]);
  o.s.spi = R(d.s[4]);
  o.s.st = R(d.s[5]);
  if (d.Q == 14) scale_rows<14>(o.s);
  else if (d.Q == 18) scale_rows<18>(o.s);
  else scale_rows<26>(o.s);
  for (int k = 0; k < 3; ++k) o.F[k] = R(F[k]);
  o.key = 0;
  if (d.Q == 14) fill_offsets<14>(o);
  else if (d.Q == 18) fill_offsets<18>(o);
  else fill_offsets<26>(o);
  return o;
}
template Domain<double> to_domain<double>(const DomainDesc&, const double*);
template Domain<float> to_domain<float>(const DomainDesc&, const double*);

void force_at(const DomainDesc& d, int64_t n, double F[3]) {
  const double c = d.period > 0.0 ? std::cos(2.0 * M_PI * (double)n / d.period) : 1.0;
  for (int k = 0; k < 3; ++k) F[k] = d.force[k] * c;
}

const char* set_faces(DomainDesc& d, const lbm_geom* g) {
  for (int f = 0; f < 6; ++f)
    if (g->face[f] < LBM_PERIODIC || g->face[f] > LBM_NEQ_PRESSURE) return "unknown face kind";
  for (int f = 0; f < 6; ++f) {
    const int n = f < 2 ? d.nx : (f < 4 ? d.ny : d.nz);
    if ((g->face[f] == LBM_NEQ_VELOCITY || g->face[f] == LBM_NEQ_PRESSURE) && n < 3)
      return "an extrapolation face needs at least 3 nodes along its axis";
  }
  int per[3];
  for (int k = 0; k < 3; ++k) {
    const bool lo = g->face[2 * k] == LBM_PERIODIC, hi = g->face[2 * k + 1] == LBM_PERIODIC;
    if (lo != hi) return "opposite faces must both be periodic or neither";
    per[k] = lo ? 1 : 0;
  }
  for (int f = 0; f < 6; ++f) {
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(g->u_wall[f][k])) return "wall velocity not finite";
    const int k = g->edge_axis[f];
    if (k == 0) continue;
    if (k < 0 || k > 3) return "edge_axis must be 0 (none) or an axis + 1";
    if (g->face[f] != LBM_MOVING_WALL) return "an edge profile needs a moving face";
    if (k - 1 == f / 2) return "an edge profile runs along an in-plane axis of its face";
    if (!std::isfinite(g->edge_scale[f][0]) || !std::isfinite(g->edge_scale[f][1]))
      return "edge scale not finite";
  }
  for (int k = 0; k < 3; ++k) d.per[k] = per[k];
  d.moving = d.sym = d.neq_vel = d.neq_pre = 0;
  for (int f = 0; f < 6; ++f) {
    if (g->face[f] == LBM_MOVING_WALL) d.moving |= 1 << f;
    if (g->face[f] == LBM_SYMMETRY) d.sym |= 1 << f;
    if (g->face[f] == LBM_NEQ_VELOCITY) d.neq_vel |= 1 << f;
    if (g->face[f] == LBM_NEQ_PRESSURE) d.neq_pre |= 1 << f;
    const bool has_u = g->face[f] == LBM_MOVING_WALL || g->face[f] == LBM_NEQ_VELOCITY;
    for (int k = 0; k < 3; ++k) d.uw[f][k] = has_u ? g->u_wall[f][k] : 0.0;
    d.edge_axis[f] = g->edge_axis[f];
    d.edge_scale[f][0] = g->edge_axis[f] ? g->edge_scale[f][0] : 1.0;
    d.edge_scale[f][1] = g->edge_axis[f] ? g->edge_scale[f][1] : 1.0;
  }
  return nullptr;
}

BlockShape default_block(int nx, int ny) {
  int bx = 32;
  while (bx < nx && bx < 128) bx *= 2;
  int by = 256 / bx;
  while (by > 1 && by / 2 >= ny) by /= 2;
  return {bx, by, 1};
}

cudaError_t launch_step_q14(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st);
cudaError_t launch_step_q18(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st);
cudaError_t launch_step_q26(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st);

cudaError_t launch_step(const DomainDesc& d, int64_t n, BlockShape b, cudaStream_t st) {
  if (d.N == 0) return cudaSuccess;
  if (d.Q == 14) return launch_step_q14(d, n, b, st);
  if (d.Q == 18) return launch_step_q18(d, n, b, st);
  if (d.Q == 26) return launch_step_q26(d, n, b, st);
  return cudaErrorInvalidValue;
}

}  // namespace lbm
