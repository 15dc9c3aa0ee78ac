// Field I/O and FP64 reductions of a single domain: equilibrium
// initialisation, canonical read-back (u, p, populations), checkpoint
// restore, and the convergence / mass / flux reductions.
#include <cmath>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

template <typename R>
Domain<R> to_domain(const DomainDesc& d, const double F[3]);

namespace {

// u and P of canonical populations fv (FP64), with the force half step.
template <int Q>
__device__ __forceinline__ void macro(const double* fv, const double F[3], double& P,
                                      double u[3]) {
  P = 0.0;
  u[0] = u[1] = u[2] = 0.0;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    P += fv[a];
    u[0] += Lattice<Q>::c(a, 0) * fv[a];
    u[1] += Lattice<Q>::c(a, 1) * fv[a];
    u[2] += Lattice<Q>::c(a, 2) * fv[a];
  }
  for (int k = 0; k < 3; ++k) u[k] += 0.5 * F[k];
}

template <int Q>
__device__ __forceinline__ double pressure_of(double P, const double u[3]) {
  // Eq. hgl with c_s^2 = 1/3
  const double cs2 = 1.0 / 3.0, w0 = Lattice<Q>::w0;
  const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return cs2 / (1.0 - w0) * (P - w0 * u2 / (2.0 * cs2));
}

struct FieldArgs {
  const double* u_in;
  const double* p_in;
  void* dst;
  const double* src;
  unsigned mask;
  int dtype;
  double F[3];
  double p_ref;
};

template <int Q, typename S, bool ODD>
__global__ void k_read(Domain<double> d, FieldArgs a) {
  const int64_t N = d.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    x = (int)(i % d.nx);
    const int64_t r = i / d.nx;
    y = (int)(r % d.ny);
    z = (int)(r / d.ny);
    double fv[Q];
    double P, u[3], p;
    if (d.solid && (d.solid[i] & kSolidCell)) {  // solid nodes report zero
      for (int b = 0; b < Q; ++b) fv[b] = 0.0;
      u[0] = u[1] = u[2] = p = 0.0;
    } else {
      get_canonical<Q, S, double, ODD>(d, static_cast<const S*>(d.f), x, y, z, fv);
      for (int b = 0; b < Q; ++b) fv[b] += 3.0 * Lattice<Q>::w(b) * a.p_ref;
      macro<Q>(fv, a.F, P, u);
      p = pressure_of<Q>(P, u);
    }
    int64_t off = 0;
    auto put = [&](int64_t k, double v) {
      if (a.dtype == LBM_DTYPE_F64) static_cast<double*>(a.dst)[k] = v;
      else static_cast<float*>(a.dst)[k] = (float)v;
    };
    if (a.mask & LBM_FIELD_U) {
      for (int k = 0; k < 3; ++k) put(off + k * N + i, u[k]);
      off += 3 * N;
    }
    if (a.mask & LBM_FIELD_P) {
      put(off + i, p);
      off += N;
    }
    if (a.mask & LBM_FIELD_POPULATIONS) {
      for (int b = 0; b < Q; ++b) put(off + b * N + i, fv[b]);
    }
  }
}

template <int Q, typename S, bool ODD>
__global__ void k_write(Domain<double> d, FieldArgs a) {
  const int64_t N = d.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % d.nx);
    const int64_t r = i / d.nx;
    const int y = (int)(r % d.ny), z = (int)(r / d.ny);
    // a solid node holds nothing (and at odd parity its canonical slots
    // hold the bounce-back values of its fluid neighbours)
    if (d.solid && (d.solid[i] & kSolidCell)) continue;
    double fv[Q];
    for (int b = 0; b < Q; ++b)
      fv[b] = a.src[b * N + i] - 3.0 * Lattice<Q>::w(b) * a.p_ref;
    put_canonical<Q, S, double, ODD>(d, static_cast<S*>(d.f), x, y, z, fv);
  }
}

template <int Q, typename S>
__global__ void k_init(Domain<double> d, FieldArgs a) {
  const int64_t N = d.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % d.nx);
    const int64_t r = i / d.nx;
    const int y = (int)(r % d.ny), z = (int)(r / d.ny);
    double u[3] = {0.0, 0.0, 0.0};
    if (a.u_in)
      for (int k = 0; k < 3; ++k) u[k] = a.u_in[k * N + i];
    const double p = (a.p_in ? a.p_in[i] : 0.0) - a.p_ref;
    const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double fv[Q];
    const bool solid = d.solid && (d.solid[i] & kSolidCell);
    // Eq. edf with lambda_a = w_a p / c_s^2 (Eq. lamda_alpha), c_s^2 = 1/3
#pragma unroll
    for (int b = 0; b < Q; ++b) {
      const double cu = Lattice<Q>::c(b, 0) * u[0] + Lattice<Q>::c(b, 1) * u[1] +
                        Lattice<Q>::c(b, 2) * u[2];
      fv[b] = solid ? 0.0 : Lattice<Q>::w(b) * (3.0 * p + 3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
    }
    put_canonical<Q, S, double, false>(d, static_cast<S*>(d.f), x, y, z, fv);
  }
}

// ---- reductions ---------------------------------------------------------------

struct ReduceArgs {
  double* u_prev;
  int have_prev;
  double* partials;
  double F[3];
  double p_ref;
  double uw[6][3];  // wall velocities in FP64 (the pair path's wall terms)
  double edge_scale[6][2];  // their edge profiles (Domain::edge_scale)
};

__device__ __forceinline__ void block_reduce(double (&v)[kNumStats], double* shm) {
  // warp level
#pragma unroll
  for (int k = 0; k < kNumStats; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_down_sync(0xffffffffu, v[k], o);
      v[k] = (k == kNumSums) ? fmax(v[k], t) : v[k] + t;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  if (lane == 0)
    for (int k = 0; k < kNumStats; ++k) shm[warp * kNumStats + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nwarps; ++w)
      for (int k = 0; k < kNumStats; ++k) {
        const double t = shm[w * kNumStats + k];
        v[k] = (k == kNumSums) ? fmax(v[k], t) : v[k] + t;
      }
  }
}

template <int Q, typename S, bool ODD>
__global__ void __launch_bounds__(kReduceThreads) k_reduce(Domain<double> d, ReduceArgs a) {
  __shared__ double shm[(kReduceThreads / 32) * kNumStats];
  double v[kNumStats];
  for (int k = 0; k < kNumStats; ++k) v[k] = 0.0;
  const int64_t N = d.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % d.nx);
    const int64_t r = i / d.nx;
    const int y = (int)(r % d.ny), z = (int)(r / d.ny);
    if (d.solid && (d.solid[i] & kSolidCell)) {  // no flow: zero in every sum
      if (a.u_prev)
        for (int k = 0; k < 3; ++k) a.u_prev[k * N + i] = 0.0;
      continue;
    }
    double fv[Q];
    get_canonical<Q, S, double, ODD>(d, static_cast<const S*>(d.f), x, y, z, fv);
    double P, u[3];
    macro<Q>(fv, a.F, P, u);
    const bool finite = isfinite(P) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
    if (!finite) {
      v[kNumSums - 1] += 1.0;
      continue;
    }
    for (int k = 0; k < 3; ++k) {
      const double up = a.have_prev ? a.u_prev[k * N + i] : 0.0;
      if (a.have_prev) v[k] += fabs(u[k] - up);
      v[3 + k] += fabs(u[k]);
      v[6 + k] += fabs(up);
      v[10 + k] += u[k];
      v[kNumSums] = fmax(v[kNumSums], fabs(u[k]));
      if (a.u_prev) a.u_prev[k * N + i] = u[k];
    }
    v[9] += P + 3.0 * (1.0 - Lattice<Q>::w0) * a.p_ref;
  }
  block_reduce(v, shm);
  if (threadIdx.x == 0)
    for (int k = 0; k < kNumStats; ++k) a.partials[blockIdx.x * kNumStats + k] = v[k];
}

// A value kept as the unevaluated pair hi + lo of FP32 numbers.  Each
// addition of an FP32 number is Knuth's TwoSum: the rounding error of
// hi + x, which it computes exactly, goes into lo.  The pair carries about
// 48 significant bits at the cost of FP32 instructions.  The reductions for
// FP32 / FP16 / BF16 storage run entirely on such pairs (a cell's P and j,
// u, the differences to the snapshot and the per-thread sums), because the
// FP64 rate of this device is a small fraction of its FP32 rate; only the
// per-thread totals are combined in FP64.  Every operation is a plain IEEE
// add or subtract in a fixed order, so results are deterministic.
struct PairSum {
  float hi = 0.0f, lo = 0.0f;
};
__device__ __forceinline__ void add_exact(PairSum& s, float x) {
  const float t = s.hi + x;
  const float xv = t - s.hi;
  const float e = (s.hi - (t - xv)) + (x - xv);
  s.hi = t;
  s.lo += e;
}
// s += p (p's low word only needs s.lo's precision)
__device__ __forceinline__ void add_pair(PairSum& s, PairSum p) {
  add_exact(s, p.hi);
  s.lo += p.lo;
}
// hi + lo with |lo| at most half an ulp of hi (Fast2Sum; |hi| >= |lo|)
__device__ __forceinline__ PairSum normalized(PairSum p) {
  const float t = p.hi + p.lo;
  return PairSum{t, p.lo - (t - p.hi)};
}
__device__ __forceinline__ PairSum negated(PairSum p) { return PairSum{-p.hi, -p.lo}; }
__device__ __forceinline__ PairSum abs_of(PairSum p) {  // p normalized
  return (p.hi < 0.0f || (p.hi == 0.0f && p.lo < 0.0f)) ? negated(p) : p;
}
__host__ __device__ inline PairSum pair_of(double x) {
  const float h = (float)x;
  return PairSum{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double value_of(PairSum s) { return (double)s.hi + (double)s.lo; }
// a > b for normalized pairs
__device__ __forceinline__ bool greater(PairSum a, PairSum b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}

// P and j of cell (x, y, z) into pairs: the stored values (exact in FP32)
// and, on odd steps, the moving-wall terms 6 w_a (c_a . u_w) of the links
// whose source is a ghost beyond a moving face, evaluated in FP64 from the
// FP64 wall velocities and added as pairs (the same canonical values that
// the FP64 path of get_canonical forms).
template <int Q, typename S, bool ODD, bool WIDE>
__device__ __forceinline__ void cell_moments(const Domain<float>& d, const S* __restrict__ f,
                                             int x, int y, int z, const double (&uw)[6][3],
                                             const double (&es)[6][2],
                                             PairSum& sP, PairSum (&sj)[3]) {
  using Ix = PopIndex<WIDE>;  // 64-bit offsets only where Q*N >= 2^31
  const int i = x + d.nx * (y + d.ny * z);
  const Ix N = (Ix)d.N;
  Links L{};
  if constexpr (ODD) L = make_links(d, x, y, z);
  [&]<int... A>(std::integer_sequence<int, A...>) {
    (
        [&] {
          constexpr int cx = Lattice<Q>::c(A, 0), cy = Lattice<Q>::c(A, 1),
                        cz = Lattice<Q>::c(A, 2);
          Ix idx = A * N + i;
          if constexpr (ODD) {
            int off, mirror;
            bool ghost;
            link_of<Q, A, -1>(L, off, ghost, mirror);
            if (!ghost) idx = opposite_mirror_rt<Q, A>(mirror) * N + i + off;
          }
          const float v = Codec<S, float>::load(f + idx);
          add_exact(sP, v);
          if constexpr (cx != 0) add_exact(sj[0], cx > 0 ? v : -v);
          if constexpr (cy != 0) add_exact(sj[1], cy > 0 ? v : -v);
          if constexpr (cz != 0) add_exact(sj[2], cz > 0 ? v : -v);
          if constexpr (ODD) {
            const int hit = link_faces<Q, A, -1>(L) & d.moving;
            if (hit) {
              int face = 0;
              while (!((hit >> face) & 1)) ++face;  // the first moving face
              double e = 1.0;  // edge profile (as edge_factor, in FP64)
              const int k = d.edge_axis[face] - 1;
              if (k >= 0) {
                if ((L.edge >> (2 * k)) & 1) e = es[face][0];
                else if ((L.edge >> (2 * k + 1)) & 1) e = es[face][1];
              }
              const double t = 6.0 * Lattice<Q>::w(A) *
                               (cx * (uw[face][0] * e) + cy * (uw[face][1] * e) +
                                cz * (uw[face][2] * e));
              const PairSum tp = pair_of(t);
              add_pair(sP, tp);
              if constexpr (cx != 0) add_pair(sj[0], cx > 0 ? tp : negated(tp));
              if constexpr (cy != 0) add_pair(sj[1], cy > 0 ? tp : negated(tp));
              if constexpr (cz != 0) add_pair(sj[2], cz > 0 ? tp : negated(tp));
            }
          }
        }(),
        ...);
  }(std::make_integer_sequence<int, Q>{});
}

// k_reduce for FP32 / FP16 / BF16 storage on PairSum arithmetic (see
// above); the statistics are those of k_reduce.  The snapshot holds each u
// component as its (hi, lo) pair in the 8 bytes of its FP64 slot.  Cells
// are numbered with 32-bit arithmetic; population offsets are 32-bit too
// unless Q*N >= 2^31 (WIDE).
template <int Q, typename S, bool ODD, bool WIDE>
__global__ void __launch_bounds__(kReduceThreads) k_reduce_pair(Domain<float> d, ReduceArgs a,
                                                                 PairSum Fh0, PairSum Fh1,
                                                                 PairSum Fh2, PairSum Pref) {
  __shared__ double shm[(kReduceThreads / 32) * kNumStats];
  PairSum sdu[3], su_abs[3], sup_abs[3], su[3], sPt, umax;
  int nonfinite = 0;
  const PairSum Fh[3] = {Fh0, Fh1, Fh2};
  // the loop counter is 64-bit only where Q*N >= 2^31 (it may pass 2^31 on
  // its last increment there); the cell index itself is below 2^31, so the
  // coordinates come from a 32-bit division
  using Ix = PopIndex<WIDE>;
  const Ix N = (Ix)d.N;
  float2* snap = reinterpret_cast<float2*>(a.u_prev);
  for (Ix i = blockIdx.x * (Ix)blockDim.x + threadIdx.x; i < N;
       i += (Ix)gridDim.x * blockDim.x) {
    const int c = (int)i;
    const int x = c % d.nx;
    const int r = c / d.nx;
    const int y = r % d.ny, z = r / d.ny;
    if (d.solid && (d.solid[i] & kSolidCell)) {  // no flow: zero in every sum
      if (a.u_prev)
        for (int k = 0; k < 3; ++k) snap[(int64_t)k * N + i] = make_float2(0.0f, 0.0f);
      continue;
    }
    PairSum sP, sj[3];
    cell_moments<Q, S, ODD, WIDE>(d, static_cast<const S*>(d.f), x, y, z, a.uw, a.edge_scale, sP,
                            sj);
    PairSum u[3];
    bool finite = isfinite(sP.hi) && isfinite(sP.lo);
    for (int k = 0; k < 3; ++k) {
      add_pair(sj[k], Fh[k]);  // u = j + F/2
      u[k] = normalized(sj[k]);
      finite = finite && isfinite(u[k].hi) && isfinite(u[k].lo);
    }
    if (!finite) {
      ++nonfinite;
      continue;
    }
    for (int k = 0; k < 3; ++k) {
      PairSum up;
      if (a.have_prev) {
        const float2 t = snap[(int64_t)k * N + i];
        up = PairSum{t.x, t.y};
        PairSum du = u[k];
        add_pair(du, negated(up));
        add_pair(sdu[k], abs_of(normalized(du)));
      }
      const PairSum ua = abs_of(u[k]);
      add_pair(su_abs[k], ua);
      add_pair(sup_abs[k], abs_of(up));
      add_pair(su[k], u[k]);
      if (greater(ua, umax)) umax = ua;
      if (a.u_prev) snap[(int64_t)k * N + i] = make_float2(u[k].hi, u[k].lo);
    }
    add_pair(sPt, normalized(sP));
    add_pair(sPt, Pref);
  }
  double v[kNumStats];
  for (int k = 0; k < 3; ++k) {
    v[k] = value_of(sdu[k]);
    v[3 + k] = value_of(su_abs[k]);
    v[6 + k] = value_of(sup_abs[k]);
    v[10 + k] = value_of(su[k]);
  }
  v[9] = value_of(sPt);
  v[kNumSums - 1] = (double)nonfinite;
  v[kNumSums] = value_of(umax);
  block_reduce(v, shm);
  if (threadIdx.x == 0)
    for (int k = 0; k < kNumStats; ++k) a.partials[blockIdx.x * kNumStats + k] = v[k];
}

// Sums the per-block partials in a fixed order (deterministic result).
__global__ void __launch_bounds__(kReduceThreads) k_reduce_final(const double* partials,
                                                                 int nblocks, double* out) {
  __shared__ double shm[(kReduceThreads / 32) * kNumStats];
  double v[kNumStats];
  for (int k = 0; k < kNumStats; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < kNumStats; ++k) {
      const double t = partials[b * kNumStats + k];
      v[k] = (k == kNumSums) ? fmax(v[k], t) : v[k] + t;
    }
  block_reduce(v, shm);
  if (threadIdx.x == 0)
    for (int k = 0; k < kNumStats; ++k) out[k] = v[k];
}

int grid_for(int64_t N) {
  int64_t g = (N + 255) / 256;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename Fn>
cudaError_t dispatch(const DomainDesc& d, Fn&& fn) {
  // fn.template operator()<Q, S>()
  if (d.Q == 14) {
    switch (d.storage) {
      case LBM_STORAGE_F64: return fn.template operator()<14, double>();
      case LBM_STORAGE_F32: return fn.template operator()<14, float>();
      case LBM_STORAGE_F16: return fn.template operator()<14, __half>();
      case LBM_STORAGE_BF16: return fn.template operator()<14, __nv_bfloat16>();
    }
  } else if (d.Q == 18) {
    switch (d.storage) {
      case LBM_STORAGE_F64: return fn.template operator()<18, double>();
      case LBM_STORAGE_F32: return fn.template operator()<18, float>();
      case LBM_STORAGE_F16: return fn.template operator()<18, __half>();
      case LBM_STORAGE_BF16: return fn.template operator()<18, __nv_bfloat16>();
    }
  } else if (d.Q == 26) {
    switch (d.storage) {
      case LBM_STORAGE_F64: return fn.template operator()<26, double>();
      case LBM_STORAGE_F32: return fn.template operator()<26, float>();
      case LBM_STORAGE_F16: return fn.template operator()<26, __half>();
      case LBM_STORAGE_BF16: return fn.template operator()<26, __nv_bfloat16>();
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_init(const DomainDesc& dd, const double* u, const double* p,
                        cudaStream_t st) {
  if (dd.N == 0) return cudaSuccess;
  const double zero[3] = {0.0, 0.0, 0.0};
  Domain<double> d = to_domain<double>(dd, zero);
  FieldArgs a{};
  a.u_in = u;
  a.p_in = p;
  a.p_ref = dd.p_ref;
  return dispatch(dd, [&]<int Q, typename S>() {
    k_init<Q, S><<<grid_for(dd.N), 256, 0, st>>>(d, a);
    return cudaGetLastError();
  });
}

cudaError_t launch_read(const DomainDesc& dd, int64_t n, unsigned mask, void* dst,
                        int dtype, cudaStream_t st) {
  if (dd.N == 0) return cudaSuccess;
  double F[3];
  force_at(dd, n, F);
  Domain<double> d = to_domain<double>(dd, F);
  FieldArgs a{};
  a.dst = dst;
  a.mask = mask;
  a.dtype = dtype;
  a.p_ref = dd.p_ref;
  for (int k = 0; k < 3; ++k) a.F[k] = F[k];
  const bool odd = n & 1;
  return dispatch(dd, [&]<int Q, typename S>() {
    if (odd) k_read<Q, S, true><<<grid_for(dd.N), 256, 0, st>>>(d, a);
    else k_read<Q, S, false><<<grid_for(dd.N), 256, 0, st>>>(d, a);
    return cudaGetLastError();
  });
}

cudaError_t launch_write(const DomainDesc& dd, int64_t n, const double* src,
                         cudaStream_t st) {
  if (dd.N == 0) return cudaSuccess;
  const double zero[3] = {0.0, 0.0, 0.0};
  Domain<double> d = to_domain<double>(dd, zero);
  FieldArgs a{};
  a.src = src;
  a.p_ref = dd.p_ref;
  const bool odd = n & 1;
  return dispatch(dd, [&]<int Q, typename S>() {
    if (odd) k_write<Q, S, true><<<grid_for(dd.N), 256, 0, st>>>(d, a);
    else k_write<Q, S, false><<<grid_for(dd.N), 256, 0, st>>>(d, a);
    return cudaGetLastError();
  });
}

cudaError_t launch_reduce(const DomainDesc& dd, int64_t n, double* u_prev, int have_prev,
                          double* partials, double* out, cudaStream_t st) {
  double F[3];
  force_at(dd, n, F);
  Domain<double> d = to_domain<double>(dd, F);
  ReduceArgs a{};
  a.u_prev = u_prev;
  a.have_prev = have_prev && u_prev != nullptr;
  a.partials = partials;
  a.p_ref = dd.p_ref;
  for (int k = 0; k < 3; ++k) a.F[k] = F[k];
  for (int face = 0; face < 6; ++face) {
    for (int k = 0; k < 3; ++k) a.uw[face][k] = dd.uw[face][k];
    for (int k = 0; k < 2; ++k) a.edge_scale[face][k] = dd.edge_scale[face][k];
  }
  int64_t g = (dd.N + kReduceThreads - 1) / kReduceThreads;
  if (g > kReduceBlocks) g = kReduceBlocks;
  if (g < 1) g = 1;
  const bool odd = n & 1;
  const Domain<float> df = to_domain<float>(dd, F);
  cudaError_t e = dispatch(dd, [&]<int Q, typename S>() {
    if constexpr (sizeof(S) <= 4) {
      const PairSum f0 = pair_of(0.5 * F[0]), f1 = pair_of(0.5 * F[1]),
                    f2 = pair_of(0.5 * F[2]);
      const PairSum pr = pair_of(3.0 * (1.0 - Lattice<Q>::w0) * dd.p_ref);
      const bool wide = (int64_t)dd.Q * dd.N >= (int64_t(1) << 31);
      auto kernel = wide ? (odd ? k_reduce_pair<Q, S, true, true> : k_reduce_pair<Q, S, false, true>)
                         : (odd ? k_reduce_pair<Q, S, true, false> : k_reduce_pair<Q, S, false, false>);
      kernel<<<(int)g, kReduceThreads, 0, st>>>(df, a, f0, f1, f2, pr);
    } else {
      if (odd) k_reduce<Q, S, true><<<(int)g, kReduceThreads, 0, st>>>(d, a);
      else k_reduce<Q, S, false><<<(int)g, kReduceThreads, 0, st>>>(d, a);
    }
    return cudaGetLastError();
  });
  if (e != cudaSuccess) return e;
  k_reduce_final<<<1, kReduceThreads, 0, st>>>(partials, (int)g, out);
  return cudaGetLastError();
}

}  // namespace lbm
