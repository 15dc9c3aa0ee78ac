// Non-equilibrium extrapolation boundaries (LBM_NEQ_VELOCITY / _PRESSURE),
// the boundary scheme the paper applies in all its simulations (Sec. 4,
// after Guo, Zheng and Shi).  The outermost node layer of such a face lies
// on the boundary; the fused step updates it like any node (its links to the
// outside read a bounce-back placeholder), then this pass replaces every
// population of every boundary node x_b:
//   f_a(x_b) = f_eq,a(p_b, u_b) + [f_a(x_f) - f_eq,a(p_f, u_f)]
// with x_f one node inward along the normal of each extrapolation face x_b
// lies on, (p_f, u_f) from f(x_f) by Eq. hgl, f_eq by Eq. edf, u_b the
// face's velocity on velocity faces (else u_f) and p_b the face's pressure
// on pressure faces (else p_f).
//
// Race freedom: x_f is never a boundary node (each extrapolation axis has at
// least 3 nodes), and in either storage layout the slots this pass reads
// (x_f's canonical populations) and writes (x_b's) are disjoint, so the
// nodes can be processed in any order in one launch.
#include <cmath>

#include "lbm_internal.h"
#include "lbm_neq.cuh"

namespace lbm {

template <typename R>
Domain<R> to_domain(const DomainDesc& d, const double F[3]);

namespace {

template <int Q, typename S, typename R, bool ODD>
__global__ void __launch_bounds__(256) k_neq(Domain<R> d, NeqArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < a.off[6]) neq_node<Q, S, R, ODD>(d, a, t);
}

template <int Q, typename S, typename R>
void launch_typed(const DomainDesc& dd, int64_t n, const NeqArgs& a, cudaStream_t st) {
  double F[3];
  force_at(dd, n, F);
  const Domain<R> d = to_domain<R>(dd, F);
  const int threads = 256, blocks = (a.off[6] + threads - 1) / threads;
  if (n & 1) k_neq<Q, S, R, true><<<blocks, threads, 0, st>>>(d, a);
  else k_neq<Q, S, R, false><<<blocks, threads, 0, st>>>(d, a);
}

}  // namespace

cudaError_t launch_neq(const DomainDesc& d, int64_t n, cudaStream_t st) {
  NeqArgs a{};
  a.vel = d.neq_vel;
  a.pre = d.neq_pre;
  if (!(a.vel | a.pre)) return cudaSuccess;
  const int64_t plane[3] = {(int64_t)d.ny * d.nz, (int64_t)d.nx * d.nz, (int64_t)d.nx * d.ny};
  a.off[0] = 0;
  for (int f = 0; f < 6; ++f) {
    const bool on = (((a.vel | a.pre) >> f) & 1) != 0;
    const int64_t next = a.off[f] + (on ? plane[f >> 1] : 0);
    if (next > (int64_t(1) << 30)) return cudaErrorInvalidValue;
    a.off[f + 1] = (int)next;
  }
  for (int f = 0; f < 6; ++f) {
    const double c = d.p_period > 0.0 ? std::cos(2.0 * M_PI * (double)n / d.p_period) : 1.0;
    a.pb[f] = d.p_face[f] + d.p_amp[f] * (d.p_period > 0.0 ? c : 0.0) - d.p_ref;
  }
  switch (d.Q * 10 + d.storage) {
    case 140: launch_typed<14, double, double>(d, n, a, st); break;
    case 141: launch_typed<14, float, float>(d, n, a, st); break;
    case 142: launch_typed<14, __half, float>(d, n, a, st); break;
    case 143: launch_typed<14, __nv_bfloat16, float>(d, n, a, st); break;
    case 180: launch_typed<18, double, double>(d, n, a, st); break;
    case 181: launch_typed<18, float, float>(d, n, a, st); break;
    case 182: launch_typed<18, __half, float>(d, n, a, st); break;
    case 183: launch_typed<18, __nv_bfloat16, float>(d, n, a, st); break;
    case 260: launch_typed<26, double, double>(d, n, a, st); break;
    case 261: launch_typed<26, float, float>(d, n, a, st); break;
    case 262: launch_typed<26, __half, float>(d, n, a, st); break;
    case 263: launch_typed<26, __nv_bfloat16, float>(d, n, a, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbm
