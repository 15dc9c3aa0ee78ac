// Allocation-free variant of the FP64 reductions (lbm_reductions_static).
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another allocator with a fixed budget (a framework's caching allocator
// that already holds the free memory), latency-critical loops that must not
// pay for cudaMalloc/cudaFree (cudaFree synchronises the whole device and
// stalls every other stream), and host code that runs where CUDA allocation
// calls are not allowed.  For them this entry point works on buffers the
// caller already owns and keeps its only scratch -- one FP64 partial sum per
// thread block plus the final statistics -- in a file-scope __device__
// array that every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "lbm_internal.h"
#include "lbm_kernels.cuh"

namespace lbm {

template <typename R>
Domain<R> to_domain(const DomainDesc& d, const double F[3]);

namespace {

constexpr int kStaticThreads = 256;
// One cell per thread and one partial per block: the static scratch bounds
// the domain at kStaticBlocks * kStaticThreads cells (= 128^3).
constexpr int kStaticBlocks = 8192;
constexpr int64_t kStaticMaxCells = int64_t(kStaticBlocks) * kStaticThreads;

// partials[kStaticBlocks][kNumStats], then the final kNumStats statistics:
// (8192 * 15 + 15) doubles = 983,160 bytes per GPU.
static __device__ __align__(256) double g_static_scratch[kStaticBlocks * kNumStats + kNumStats];

// Device addresses of g_static_scratch, looked up once per device.  In host
// code the array's name is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

template <int Q>
__device__ __forceinline__ void cell_stats(const double* fv, const double F[3], double& P,
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

// Sums (max for the last entry) of v over the block; result in thread 0.
__device__ __forceinline__ void block_sum(double (&v)[kNumStats], double* shm) {
#pragma unroll
  for (int k = 0; k < kNumStats; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double t = __shfl_down_sync(0xffffffffu, v[k], o);
      v[k] = (k == kNumSums) ? fmax(v[k], t) : v[k] + t;
    }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
    for (int k = 0; k < kNumStats; ++k) shm[warp * kNumStats + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      for (int k = 0; k < kNumStats; ++k) {
        const double t = shm[w * kNumStats + k];
        v[k] = (k == kNumSums) ? fmax(v[k], t) : v[k] + t;
      }
}

struct StaticArgs {
  double* scratch;  // device address of g_static_scratch
  double* u_prev;   // caller's 3N snapshot, or null
  int have_prev;
  double F[3];
  double p_ref;
};

// One cell per thread; block b writes partial b of the scratch.
template <int Q, typename S, bool ODD>
__global__ void __launch_bounds__(kStaticThreads) k_reduce_static(Domain<double> d, StaticArgs a) {
  __shared__ double shm[(kStaticThreads / 32) * kNumStats];
  double v[kNumStats];
  for (int k = 0; k < kNumStats; ++k) v[k] = 0.0;
  const int64_t N = d.N;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) {
    const int x = (int)(i % d.nx);
    const int64_t r = i / d.nx;
    const int y = (int)(r % d.ny), z = (int)(r / d.ny);
    double fv[Q];
    get_canonical<Q, S, double, ODD>(d, static_cast<const S*>(d.f), x, y, z, fv);
    double P, u[3];
    cell_stats<Q>(fv, a.F, P, u);
    if (!(isfinite(P) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]))) {
      v[kNumSums - 1] = 1.0;
    } else {
      for (int k = 0; k < 3; ++k) {
        const double up = (a.u_prev && a.have_prev) ? a.u_prev[k * N + i] : 0.0;
        if (a.u_prev && a.have_prev) v[k] = fabs(u[k] - up);
        v[3 + k] = fabs(u[k]);
        v[6 + k] = fabs(up);
        v[10 + k] = u[k];
        v[kNumSums] = fmax(v[kNumSums], fabs(u[k]));
        if (a.u_prev) a.u_prev[k * N + i] = u[k];
      }
      v[9] = P + 3.0 * (1.0 - Lattice<Q>::w0) * a.p_ref;
    }
  }
  block_sum(v, shm);
  if (threadIdx.x == 0)
    for (int k = 0; k < kNumStats; ++k) a.scratch[blockIdx.x * kNumStats + k] = v[k];
}

// Sums the first `nblocks` partials in a fixed order into the stats slot.
__global__ void __launch_bounds__(kStaticThreads) k_reduce_static_final(double* scratch,
                                                                        int nblocks) {
  __shared__ double shm[(kStaticThreads / 32) * kNumStats];
  double v[kNumStats];
  for (int k = 0; k < kNumStats; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < kNumStats; ++k) {
      const double t = scratch[b * kNumStats + k];
      v[k] = (k == kNumSums) ? fmax(v[k], t) : v[k] + t;
    }
  block_sum(v, shm);
  if (threadIdx.x == 0)
    for (int k = 0; k < kNumStats; ++k)
      scratch[kStaticBlocks * kNumStats + k] = v[k];
}

int static_fail(int code, const std::string& msg) {
  set_last_error(msg);  // reported by lbm_last_error()
  return code;
}

}  // namespace

}  // namespace lbm

using namespace lbm;

extern "C" int lbm_reductions_static(const lbm_desc* desc, const lbm_geom* geom,
                                     const lbm_params* params, int64_t step,
                                     const void* populations, double* u_prev,
                                     int64_t prev_step, lbm_stats* out, void* cuda_stream) {
  if (!desc || !geom || !params || !populations || !out)
    return static_fail(LBM_EINVAL, "null argument");
  if (desc->Q != 14 && desc->Q != 18 && desc->Q != 26)
    return static_fail(LBM_EINVAL, "Q must be 14, 18 or 26");
  if (desc->nx < 1 || desc->ny < 1 || desc->nz < 1 || step < 0)
    return static_fail(LBM_EINVAL, "grid sizes must be >= 1 and step >= 0");
  if (desc->storage < LBM_STORAGE_F64 || desc->storage > LBM_STORAGE_BF16)
    return static_fail(LBM_EINVAL, "unknown storage type");
  const int64_t N = (int64_t)desc->nx * desc->ny * desc->nz;
  if (N > kStaticMaxCells)
    return static_fail(LBM_EINVAL,
                       "domain has " + std::to_string(N) + " cells; the static scratch of "
                       "lbm_reductions_static holds at most " +
                           std::to_string(kStaticMaxCells) + " cells");
  DomainDesc dd{};
  dd.Q = desc->Q;
  dd.nx = desc->nx;
  dd.ny = desc->ny;
  dd.nz = desc->nz;
  dd.storage = desc->storage;
  dd.N = N;
  if (const char* why = set_faces(dd, geom)) return static_fail(LBM_EINVAL, why);
  dd.f = const_cast<void*>(populations);
  for (int k = 0; k < 3; ++k) dd.force[k] = params->force[k];
  dd.period = params->force_period;
  dd.p_ref = params->p_ref;
  double F[3];
  force_at(dd, step, F);

  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess)
    return static_fail(LBM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  Domain<double> d = to_domain<double>(dd, F);
  StaticArgs a{};
  a.scratch = scratch;
  a.u_prev = u_prev;
  a.have_prev = (u_prev && prev_step >= 0) ? 1 : 0;
  a.p_ref = dd.p_ref;
  for (int k = 0; k < 3; ++k) a.F[k] = F[k];
  const int blocks = (int)((N + kStaticThreads - 1) / kStaticThreads);
  const bool odd = step & 1;
  auto launch = [&]<int Q, typename S>() {
    if (odd) k_reduce_static<Q, S, true><<<blocks, kStaticThreads, 0, st>>>(d, a);
    else k_reduce_static<Q, S, false><<<blocks, kStaticThreads, 0, st>>>(d, a);
  };
  if (dd.Q == 14) {
    switch (dd.storage) {
      case LBM_STORAGE_F64: launch.template operator()<14, double>(); break;
      case LBM_STORAGE_F32: launch.template operator()<14, float>(); break;
      case LBM_STORAGE_F16: launch.template operator()<14, __half>(); break;
      default: launch.template operator()<14, __nv_bfloat16>(); break;
    }
  } else if (dd.Q == 18) {
    switch (dd.storage) {
      case LBM_STORAGE_F64: launch.template operator()<18, double>(); break;
      case LBM_STORAGE_F32: launch.template operator()<18, float>(); break;
      case LBM_STORAGE_F16: launch.template operator()<18, __half>(); break;
      default: launch.template operator()<18, __nv_bfloat16>(); break;
    }
  } else {
    switch (dd.storage) {
      case LBM_STORAGE_F64: launch.template operator()<26, double>(); break;
      case LBM_STORAGE_F32: launch.template operator()<26, float>(); break;
      case LBM_STORAGE_F16: launch.template operator()<26, __half>(); break;
      default: launch.template operator()<26, __nv_bfloat16>(); break;
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return static_fail(LBM_ECUDA, std::string("reduction kernel: ") + cudaGetErrorString(e));
  k_reduce_static_final<<<1, kStaticThreads, 0, st>>>(scratch, blocks);
  e = cudaGetLastError();
  double s[kNumStats];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s, scratch + kStaticBlocks * kNumStats, sizeof s,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return static_fail(LBM_ECUDA, std::string("static reduction: ") + cudaGetErrorString(e));
  out->step = step;
  out->prev_step = a.have_prev ? prev_step : -1;
  for (int k = 0; k < 3; ++k) {
    out->sum_abs_du[k] = s[k];
    out->sum_abs_u[k] = s[3 + k];
    out->sum_abs_u_prev[k] = s[6 + k];
    out->sum_u[k] = s[10 + k];
  }
  out->sum_P = s[9];
  out->nonfinite = (int64_t)s[kNumSums - 1];
  out->max_abs_u = s[kNumSums];
  return LBM_OK;
}

